// Device form of the reduced-model construction (rom_build_gpu), FP64.
// Included by rom_build.cu inside its anonymous namespace (it uses FineSys
// and PencilSolver).
//
// The block Krylov basis of Sec. III (start block (psi0 R + F)^{-1} B B_in,
// operator (psi0 R + F)^{-1} R), its block orthogonalisation and the
// congruences of Eq. (12) run on the device; the host keeps the banded
// Cholesky factorisation of the Hz Schur complement (done once), the
// eigen-decompositions of the small Gram matrices and everything after the
// congruences (Eq. (27), the report).  All matrices on the device are
// column-major, one column per Krylov vector.
//
// Orthonormalisation uses Gram matrices instead of Householder QR:
// W <- W - Q (Q^T W) twice (classical Gram-Schmidt, re-orthogonalised), then
// W^T W = V diag(s^2) V^T, U = W V diag(1/s) for the kept directions, and one
// Cholesky-QR pass U <- U chol(U^T U)^{-1}.  One Gram matrix resolves s only
// down to ~1e-8 of the largest, so the directions below 1e-7 are found in a
// second stage on the remainder X - U U^T X (gram_basis); the deflation
// tolerance (1e-12 relative) and the singular-value gap rule for a block cut
// to fit q/2 are the host build's.
#pragma once

#include <cuda_runtime.h>

// ---------------------------------------------------------------- kernels

// T = X_E / a11 (first step of the pencil solve; pencil_h_kernel then forms
// X_H - c K^T T).  Column c of X at X + c * N.
__global__ void pencil_pre_kernel(const double* __restrict__ X, double* __restrict__ T, int N, int nE, int m,
                                  const double* __restrict__ a11) {
  const long long tot = (long long)m * nE;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / nE), e = (int)(k - (long long)col * nE);
    T[(size_t)col * nE + e] = X[(size_t)col * N + e] / a11[e];
  }
}

__global__ void pencil_h_kernel(double* __restrict__ X, const double* __restrict__ T, int N, int nE, int nH,
                                int m, const int* __restrict__ kte, const double* __restrict__ ktv, double c) {
  const long long tot = (long long)m * nH;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / nH), h = (int)(k - (long long)col * nH);
    const double* t = T + (size_t)col * nE;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) s += ktv[(size_t)q * nH + h] * t[kte[(size_t)q * nH + h]];
    X[(size_t)col * N + nE + h] -= c * s;
  }
}

// Banded Cholesky solve L L^T x = b for every column's Hz part, one warp per
// column; the last bw + 1 solved values of a sweep sit in a shared ring.
// L is row-major in (bw + 1) slots per row: L(i, j) at L[i (bw+1) + i - j].
__global__ void band_solve_kernel(double* __restrict__ X, int N, int nE, int nH, int m,
                                  const double* __restrict__ L, int bw) {
  extern __shared__ double ring_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + warp;
  if (col >= m) return;
  double* ring = ring_all + (size_t)warp * (bw + 1);
  double* x = X + (size_t)col * N + nE;
  const unsigned FULL = 0xffffffffu;
  const int W = bw + 1;
  for (int i = 0; i < nH; ++i) {   // L y = b
    double s = 0.0;
    const int k0 = max(0, i - bw);
    for (int k = k0 + lane; k < i; k += 32) s += L[(size_t)i * W + (i - k)] * ring[k % W];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) {
      const double y = (x[i] - s) / L[(size_t)i * W];
      ring[i % W] = y;
      x[i] = y;
    }
    __syncwarp();
  }
  for (int i = nH - 1; i >= 0; --i) {   // L^T x = y
    double s = 0.0;
    const int k1 = min(nH - 1, i + bw);
    for (int k = i + 1 + lane; k <= k1; k += 32) s += L[(size_t)k * W + (k - i)] * ring[k % W];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) {
      const double v = (x[i] - s) / L[(size_t)i * W];
      ring[i % W] = v;
      x[i] = v;
    }
    __syncwarp();
  }
}

// X_E <- T + c K X_H / a11 (second half of the pencil solve).
__global__ void pencil_post_kernel(double* __restrict__ X, const double* __restrict__ T, int N, int nE,
                                   int m, const double* __restrict__ a11, const int* __restrict__ kh,
                                   const double* __restrict__ kv, double c) {
  const long long tot = (long long)m * nE;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / nE), e = (int)(k - (long long)col * nE);
    const double* h = X + (size_t)col * N + nE;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int hi = kh[(size_t)q * nE + e];
      if (hi >= 0) s += kv[(size_t)q * nE + e] * h[hi];
    }
    X[(size_t)col * N + e] = T[(size_t)col * nE + e] + c * s / a11[e];
  }
}

// Y = R X at dt: Y_E = D_eps/dt X_E - K X_H / 2,  Y_H = -K^T X_E / 2 + D_mu/dt X_H.
__global__ void r_apply_kernel(const double* __restrict__ X, double* __restrict__ Y, int N, int nE, int nH,
                               int m, double dt, const double* __restrict__ deps, const double* __restrict__ dmu,
                               const int* __restrict__ kh, const double* __restrict__ kv,
                               const int* __restrict__ kte, const double* __restrict__ ktv) {
  const long long tot = (long long)m * N;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / N), r = (int)(k - (long long)col * N);
    const double* x = X + (size_t)col * N;
    double v;
    if (r < nE) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int hi = kh[(size_t)q * nE + r];
        if (hi >= 0) s += kv[(size_t)q * nE + r] * x[nE + hi];
      }
      v = deps[r] / dt * x[r] - 0.5 * s;
    } else {
      const int h = r - nE;
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) s += ktv[(size_t)q * nH + h] * x[kte[(size_t)q * nH + h]];
      v = -0.5 * s + dmu[h] / dt * x[r];
    }
    Y[(size_t)col * N + r] = v;
  }
}

// Y = K X for X on the Hz unknowns (nH x m, leading dimension ldx) into Y (nE x m).
__global__ void k_apply_kernel(const double* __restrict__ X, int ldx, double* __restrict__ Y, int nE, int m,
                               const int* __restrict__ kh, const double* __restrict__ kv) {
  const long long tot = (long long)m * nE;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / nE), e = (int)(k - (long long)col * nE);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int hi = kh[(size_t)q * nE + e];
      if (hi >= 0) s += kv[(size_t)q * nE + e] * X[(size_t)col * ldx + hi];
    }
    Y[(size_t)col * nE + e] = s;
  }
}

// Y = diag(d) X (rows), both leading dimension n.
__global__ void scale_rows_kernel(const double* __restrict__ X, int ldx, double* __restrict__ Y, int n, int m,
                                  const double* __restrict__ d) {
  const long long tot = (long long)m * n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    const int col = (int)(k / n), r = (int)(k - (long long)col * n);
    Y[(size_t)col * n + r] = d[r] * X[(size_t)col * ldx + r];
  }
}

// Partial products P[s] = A(rows of chunk s)^T B(rows of chunk s), 32 x 32
// output tiles, each thread 2 x 2 outputs; A is n x ka (lda), B n x kb (ldb).
constexpr int kGemmChunk = 4096;
__global__ void __launch_bounds__(256) gemm_tn_partial_kernel(const double* __restrict__ A, int lda,
                                                              const double* __restrict__ B, int ldb, int n,
                                                              int ka, int kb, double* __restrict__ P) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int ti = blockIdx.x * 32, tj = blockIdx.y * 32, s = blockIdx.z;
  const int r0 = s * kGemmChunk, r1 = min(n, r0 + kGemmChunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int rr = e & 31, cc = e >> 5;
      const int r = rb + rr;
      As[rr][cc] = (r < r1 && ti + cc < ka) ? A[(size_t)(ti + cc) * lda + r] : 0.0;
      Bs[rr][cc] = (r < r1 && tj + cc < kb) ? B[(size_t)(tj + cc) * ldb + r] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const double a0 = As[rr][2 * ty], a1 = As[rr][2 * ty + 1];
      const double b0 = Bs[rr][2 * tx], b1 = Bs[rr][2 * tx + 1];
      c00 += a0 * b0;
      c01 += a0 * b1;
      c10 += a1 * b0;
      c11 += a1 * b1;
    }
    __syncthreads();
  }
  double* Ps = P + (size_t)s * ka * kb;   // column-major ka x kb
  const int i0 = ti + 2 * ty, j0 = tj + 2 * tx;
  if (i0 < ka && j0 < kb) Ps[(size_t)j0 * ka + i0] = c00;
  if (i0 < ka && j0 + 1 < kb) Ps[(size_t)(j0 + 1) * ka + i0] = c01;
  if (i0 + 1 < ka && j0 < kb) Ps[(size_t)j0 * ka + i0 + 1] = c10;
  if (i0 + 1 < ka && j0 + 1 < kb) Ps[(size_t)(j0 + 1) * ka + i0 + 1] = c11;
}

// C = sum over chunks of P, in chunk order.
__global__ void gemm_reduce_kernel(const double* __restrict__ P, int nsplit, int cnt, double* __restrict__ C) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < nsplit; ++s) v += P[(size_t)s * cnt + k];
    C[k] = v;
  }
}

// C = alpha A B + beta C with A n x k (lda), B k x mc (ldb), C n x mc (ldc);
// 64 x 32 output tiles, each thread 4 x 2 outputs.
__global__ void __launch_bounds__(256) gemm_nn_kernel(const double* __restrict__ A, int lda,
                                                      const double* __restrict__ B, int ldb,
                                                      double* __restrict__ C, int ldc, int n, int k, int mc,
                                                      double alpha, double beta) {
  __shared__ double As[32][65];
  __shared__ double Bs[32][33];
  const int ti = blockIdx.x * 64, tj = blockIdx.y * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;   // rows ty*4.., cols tx*2..
  double acc[4][2] = {};
  for (int kb = 0; kb < k; kb += 32) {
    for (int e = tid; e < 64 * 32; e += 256) {
      const int rr = e & 63, kk = e >> 6;
      As[kk][rr] = (ti + rr < n && kb + kk < k) ? A[(size_t)(kb + kk) * lda + ti + rr] : 0.0;
    }
    for (int e = tid; e < 32 * 32; e += 256) {
      const int kk = e & 31, cc = e >> 5;
      Bs[kk][cc] = (kb + kk < k && tj + cc < mc) ? B[(size_t)(tj + cc) * ldb + kb + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double a = As[kk][4 * ty + u];
        acc[u][0] += a * b0;
        acc[u][1] += a * b1;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = ti + 4 * ty + u, c = tj + 2 * tx + v;
      if (r < n && c < mc) {
        double* p = C + (size_t)c * ldc + r;
        *p = alpha * acc[u][v] + (beta == 0.0 ? 0.0 : beta * *p);
      }
    }
}

// ---------------------------------------------------------------- host side

struct GpuArena {
  std::vector<void*> ptrs;
  ~GpuArena() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  template <class T>
  T* put(const T* h, size_t n) {
    T* d = get<T>(n);
    if (n && cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) throw std::bad_alloc();
    return d;
  }
};

struct GpuBuild {
  cudaStream_t st;
  GpuArena ar;
  int N, nE, nH, bw;
  double* d_eps;
  double* d_sig;
  double* d_mu;
  double* a11;
  double* L;
  int* kh;
  double* kv;
  int* kte;
  double* ktv;
  double* part = nullptr;   // split-K partials
  size_t part_cap = 0;
  double* cbuf = nullptr;   // reduced product
  size_t cbuf_cap = 0;

  unsigned grid(long long work) const { return (unsigned)std::min<long long>(4096, (work + 255) / 256); }

  static void check(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
  }

  // C (ka x kb, column-major, host) = A^T B over n rows.
  Mat gram(const double* A, int lda, const double* B, int ldb, int n, int ka, int kb) {
    const int nsplit = (n + kGemmChunk - 1) / kGemmChunk;
    const size_t need = (size_t)nsplit * ka * kb;
    if (need > part_cap) {
      part = ar.get<double>(need);
      part_cap = need;
    }
    if ((size_t)ka * kb > cbuf_cap) {
      cbuf = ar.get<double>((size_t)ka * kb);
      cbuf_cap = (size_t)ka * kb;
    }
    double* C = cbuf;
    dim3 g((ka + 31) / 32, (kb + 31) / 32, nsplit);
    gemm_tn_partial_kernel<<<g, 256, 0, st>>>(A, lda, B, ldb, n, ka, kb, part);
    gemm_reduce_kernel<<<grid((long long)ka * kb), 256, 0, st>>>(part, nsplit, ka * kb, C);
    check("rom_build_gpu: kernel launch failed");
    std::vector<double> h((size_t)ka * kb);
    if (cudaMemcpyAsync(h.data(), C, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      throw std::runtime_error("rom_build_gpu: device copy failed");
    Mat M(ka, kb);
    for (int j = 0; j < kb; ++j)
      for (int i = 0; i < ka; ++i) M(i, j) = h[(size_t)j * ka + i];
    return M;
  }

  // C (n x mc, ldc) = alpha A (n x k, lda) B + beta C, B given on the host (k x mc).
  void mul(const double* A, int lda, const Mat& Bh, double* C, int ldc, int n, double alpha, double beta) {
    const int k = Bh.r, mc = Bh.c;
    if (k == 0 || mc == 0) return;
    std::vector<double> b((size_t)k * mc);
    for (int j = 0; j < mc; ++j)
      for (int i = 0; i < k; ++i) b[(size_t)j * k + i] = Bh(i, j);
    double* B = ar.put(b.data(), b.size());
    dim3 g((n + 63) / 64, (mc + 31) / 32);
    gemm_nn_kernel<<<g, 256, 0, st>>>(A, lda, B, k, C, ldc, n, k, mc, alpha, beta);
  }

  // X <- (psi0 R + F)^{-1} X, X N x m column-major.
  void pencil_solve(double* X, int m, double psi0, double* T) {
    pencil_pre_kernel<<<grid((long long)m * nE), 256, 0, st>>>(X, T, N, nE, m, a11);
    pencil_h_kernel<<<grid((long long)m * nH), 256, 0, st>>>(X, T, N, nE, nH, m, kte, ktv, 0.5 * (1.0 - psi0));
    // warps per block so that their rings fit the default 48 KB of shared memory
    const size_t ring = sizeof(double) * (bw + 1);
    if (ring > 48 * 1024) throw std::runtime_error("rom_build_gpu: fine region wider than 6143 cells");
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(4, (48 * 1024) / ring));
    band_solve_kernel<<<(m + wpb - 1) / wpb, 32 * wpb, ring * wpb, st>>>(X, N, nE, nH, m, L, bw);
    pencil_post_kernel<<<grid((long long)m * nE), 256, 0, st>>>(X, T, N, nE, m, a11, kh, kv, 0.5 * (psi0 + 1.0));
    check("rom_build_gpu: kernel launch failed");
  }
};

// Orthonormal basis of the leading directions of W (n x m, column-major,
// leading dimension ld) with singular values above rel * ref, in decreasing
// order, written over the first columns of W; returns the singular values
// kept (all of them, the caller may cut).
std::vector<double> gram_svd(GpuBuild& g, double* W, int ld, int n, int m, double rel, double ref, Mat& V) {
  Mat G = g.gram(W, ld, W, ld, n, m, m);
  std::vector<double> w;
  Mat E;
  la::eig_sym(G, w, E);   // ascending
  std::vector<double> s;
  std::vector<int> idx;
  for (int i = m - 1; i >= 0; --i) {
    const double sv = std::sqrt(std::max(w[i], 0.0));
    if (!(sv > rel * ref)) break;
    s.push_back(sv);
    idx.push_back(i);
  }
  V = Mat(m, (int)idx.size());
  for (int c = 0; c < (int)idx.size(); ++c)
    for (int r = 0; r < m; ++r) V(r, c) = E(r, idx[c]);
  return s;
}

// U <- U chol(U^T U)^{-1} (one Cholesky-QR pass) on n x k columns.
void chol_qr(GpuBuild& g, double* U, int ld, int n, int k, double* tmp) {
  if (k == 0) return;
  Mat G = g.gram(U, ld, U, ld, n, k, k);
  // G = R^T R with R upper triangular; U <- U R^{-1}
  Mat R(k, k);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j; ++i) {
      double s = G(i, j);
      for (int t = 0; t < i; ++t) s -= R(t, i) * R(t, j);
      if (i == j) {
        if (!(s > 0.0)) throw std::runtime_error("rom_build_gpu: Cholesky-QR lost positive definiteness");
        R(i, i) = std::sqrt(s);
      } else {
        R(i, j) = s / R(i, i);
      }
    }
  }
  Mat Ri(k, k);   // R^{-1}, upper triangular
  for (int j = 0; j < k; ++j) {
    Ri(j, j) = 1.0 / R(j, j);
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int t = i + 1; t <= j; ++t) s += R(i, t) * Ri(t, j);
      Ri(i, j) = -s / R(i, i);
    }
  }
  g.mul(U, ld, Ri, tmp, n, n, 1.0, 0.0);
  cudaMemcpy2DAsync(U, sizeof(double) * ld, tmp, sizeof(double) * n, sizeof(double) * n, k,
                    cudaMemcpyDeviceToDevice, g.st);
}

// Rank-revealing orthonormal basis from Gram matrices, in two stages.  X is
// n x m (leading dimension ld); the result U (n x kept, leading dimension n)
// spans X's left singular directions with s > rel * ref (ref <= 0: the
// largest s), in decreasing order of s.  Stage 1 takes the directions a Gram
// matrix resolves (s > 1e-7 s_max); stage 2 removes them from X and repeats
// on the remainder, whose own Gram matrix resolves s down to ~1e-15 s_max.
// R is n x m scratch, Y n x m scratch for Cholesky-QR.
std::vector<double> gram_basis(GpuBuild& g, const double* X, int ld, int n, int m, double rel, double ref,
                               double* U, double* R, double* Y) {
  std::vector<double> out;
  Mat V;
  std::vector<double> s1 = gram_svd(g, const_cast<double*>(X), ld, n, m, 0.0, 0.0, V);
  if (s1.empty()) return out;
  const double smax = s1[0];
  const double thr = rel * (ref > 0 ? ref : smax);
  int k1 = 0;
  while (k1 < (int)s1.size() && s1[k1] > std::max(thr, 1e-7 * smax)) ++k1;
  if (k1 == 0) return out;
  Mat Vs(m, k1);
  for (int c = 0; c < k1; ++c)
    for (int r = 0; r < m; ++r) Vs(r, c) = V(r, c) / s1[c];
  g.mul(X, ld, Vs, U, n, n, 1.0, 0.0);
  chol_qr(g, U, n, n, k1, Y);
  out.assign(s1.begin(), s1.begin() + k1);
  if (!(thr < 1e-7 * smax) || k1 >= m) return out;
  // stage 2: R = X - U U^T X (twice), then its Gram basis
  cudaMemcpy2DAsync(R, sizeof(double) * n, X, sizeof(double) * ld, sizeof(double) * n, m,
                    cudaMemcpyDeviceToDevice, g.st);
  for (int pass = 0; pass < 2; ++pass) {
    Mat C = g.gram(U, n, R, n, n, k1, m);
    g.mul(U, n, C, R, n, n, -1.0, 1.0);
  }
  Mat V2;
  std::vector<double> s2 = gram_svd(g, R, n, n, m, 0.0, 0.0, V2);
  int k2 = 0;
  while (k2 < (int)s2.size() && s2[k2] > thr) ++k2;
  k2 = std::min(k2, m - k1);
  if (k2 == 0) return out;
  Mat Vs2(m, k2);
  for (int c = 0; c < k2; ++c)
    for (int r = 0; r < m; ++r) Vs2(r, c) = V2(r, c) / s2[c];
  double* U2 = U + (size_t)k1 * n;
  g.mul(R, n, Vs2, U2, n, n, 1.0, 0.0);
  chol_qr(g, U2, n, n, k2, Y);
  Mat C = g.gram(U, n, U2, n, n, k1, k2);   // re-orthogonalise against stage 1
  g.mul(U, n, C, U2, n, n, -1.0, 1.0);
  chol_qr(g, U2, n, n, k2, Y);
  out.insert(out.end(), s2.begin(), s2.begin() + k2);
  return out;
}

// V1, V2 and the Eq. (12) blocks of model m on the device (module header).
void gpu_blocks(const FineSys& f, const PencilSolver& ps, double psi0, double dt_b, const Mat& W0h, int k,
                double tol, cudaStream_t st, rom_model* m) {
  GpuBuild g;
  g.st = st;
  g.nE = f.nE, g.nH = f.nH, g.N = f.nE + f.nH, g.bw = ps.S.bw;
  const int N = g.N, nE = f.nE, nH = f.nH;
  g.d_eps = g.ar.put(f.d_eps.data(), nE);
  g.d_sig = g.ar.put(f.d_sig.data(), nE);
  g.d_mu = g.ar.put(f.d_mu.data(), nH);
  g.a11 = g.ar.put(ps.a11.data(), nE);
  g.L = g.ar.put(ps.S.a.data(), ps.S.a.size());
  {
    std::vector<int> kh(2 * (size_t)nE), kte(4 * (size_t)nH);
    std::vector<double> kv(2 * (size_t)nE), ktv(4 * (size_t)nH);
    for (int q = 0; q < 2; ++q)
      for (int e = 0; e < nE; ++e) kh[(size_t)q * nE + e] = f.k_h[q][e], kv[(size_t)q * nE + e] = f.k_v[q][e];
    for (int q = 0; q < 4; ++q)
      for (int h = 0; h < nH; ++h) kte[(size_t)q * nH + h] = f.kt_e[q][h], ktv[(size_t)q * nH + h] = f.kt_v[q][h];
    g.kh = g.ar.put(kh.data(), kh.size());
    g.kv = g.ar.put(kv.data(), kv.size());
    g.kte = g.ar.put(kte.data(), kte.size());
    g.ktv = g.ar.put(ktv.data(), ktv.size());
  }
  const int mw = W0h.c;
  const int mmax = std::max(mw, 1);
  double* W = g.ar.get<double>((size_t)N * mmax);
  double* Y = g.ar.get<double>((size_t)N * std::max(mmax, k));   // Cholesky-QR scratch
  double* Ub = g.ar.get<double>((size_t)N * mmax);                 // a block's basis
  double* Rs = g.ar.get<double>((size_t)N * std::max(mmax, k));   // residual of stage 2
  double* T = g.ar.get<double>((size_t)nE * mmax);
  double* Q = g.ar.get<double>((size_t)N * std::max(k, 1));
  {
    std::vector<double> w((size_t)N * mw);
    for (int j = 0; j < mw; ++j)
      for (int i = 0; i < N; ++i) w[(size_t)j * N + i] = W0h(i, j);
    cudaMemcpyAsync(W, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  g.pencil_solve(W, mw, psi0, T);
  int qc = 0, wc = mw;
  while (qc < k && wc > 0) {
    // reference norm of the block before it is orthogonalised
    Mat Vr;
    std::vector<double> s0 = gram_svd(g, W, N, N, wc, 0.0, 0.0, Vr);
    const double ref = s0.empty() ? 0.0 : s0[0];
    if (!(ref > 0.0)) break;
    for (int pass = 0; pass < 2 && qc > 0; ++pass) {   // W <- W - Q (Q^T W)
      Mat C = g.gram(Q, N, W, N, N, qc, wc);
      g.mul(Q, N, C, W, N, N, -1.0, 1.0);
    }
    std::vector<double> s = gram_basis(g, W, N, N, wc, tol, ref, Ub, Rs, Y);
    int keep = (int)s.size();
    if (keep == 0) break;
    int take = std::min(keep, k - qc);
    const bool truncated = take < keep;
    if (truncated) {   // cut at a singular-value gap (relative 1e-8), as the host build
      while (take > 0 && s[take - 1] - s[take] <= 1e-8 * s[take - 1]) --take;
      if (take == 0) break;
    }
    double* U = Q + (size_t)qc * N;
    cudaMemcpyAsync(U, Ub, sizeof(double) * N * take, cudaMemcpyDeviceToDevice, st);
    if (qc > 0) {   // one more projection against the earlier blocks, then re-normalise
      Mat C = g.gram(Q, N, U, N, N, qc, take);
      g.mul(Q, N, C, U, N, N, -1.0, 1.0);
      chol_qr(g, U, N, N, take, Y);
    }
    qc += take;
    if (truncated || qc >= k) break;
    // next block: (psi0 R + F)^{-1} R U
    r_apply_kernel<<<g.grid((long long)take * N), 256, 0, st>>>(U, W, N, nE, nH, take, dt_b, g.d_eps, g.d_mu,
                                                                 g.kh, g.kv, g.kte, g.ktv);
    wc = take;
    g.pencil_solve(W, wc, psi0, T);
  }
  // V1 = orth(E rows of Q), V2 = orth(H rows of Q)
  double* V1 = g.ar.get<double>((size_t)nE * std::max(qc, 1));
  double* V2 = g.ar.get<double>((size_t)nH * std::max(qc, 1));
  auto orth_rows = [&](const double* Qp, int n, double* out) -> int {
    return (int)gram_basis(g, Qp, N, n, qc, tol, 0.0, out, Rs, Y).size();
  };
  const int qE = orth_rows(Q, nE, V1);
  const int qH = orth_rows(Q + nE, nH, V2);
  // Eq. (12) blocks by congruence
  double* DV = g.ar.get<double>((size_t)N * std::max(std::max(qE, qH), 1));
  scale_rows_kernel<<<g.grid((long long)qE * nE), 256, 0, st>>>(V1, nE, DV, nE, qE, g.d_eps);
  m->R11 = g.gram(V1, nE, DV, nE, nE, qE, qE);
  scale_rows_kernel<<<g.grid((long long)qE * nE), 256, 0, st>>>(V1, nE, DV, nE, qE, g.d_sig);
  m->Sig = g.gram(V1, nE, DV, nE, nE, qE, qE);
  scale_rows_kernel<<<g.grid((long long)qH * nH), 256, 0, st>>>(V2, nH, DV, nH, qH, g.d_mu);
  m->R22 = g.gram(V2, nH, DV, nH, nH, qH, qH);
  k_apply_kernel<<<g.grid((long long)qH * nE), 256, 0, st>>>(V2, nH, DV, nE, qH, g.kh, g.kv);
  m->Kt = g.gram(V1, nE, DV, nE, nE, qE, qH);
  // symmetrise the Gram-type blocks (their two triangles come from one sum)
  for (Mat* A : {&m->R11, &m->Sig, &m->R22})
    for (int i = 0; i < A->r; ++i)
      for (int j = i + 1; j < A->c; ++j) (*A)(i, j) = (*A)(j, i) = 0.5 * ((*A)(i, j) + (*A)(j, i));
  // bases to the host (row-major)
  std::vector<double> h1((size_t)nE * qE), h2((size_t)nH * qH);
  cudaMemcpyAsync(h1.data(), V1, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(h2.data(), V2, sizeof(double) * h2.size(), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) throw std::runtime_error("rom_build_gpu: device failure");
  m->V1 = Mat(nE, qE);
  m->V2 = Mat(nH, qH);
  for (int j = 0; j < qE; ++j)
    for (int i = 0; i < nE; ++i) m->V1(i, j) = h1[(size_t)j * nE + i];
  for (int j = 0; j < qH; ++j)
    for (int i = 0; i < nH; ++i) m->V2(i, j) = h2[(size_t)j * nH + i];
  m->qE = qE;
  m->qH = qH;
}
