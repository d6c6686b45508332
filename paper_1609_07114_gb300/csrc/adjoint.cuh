// Discrete adjoint of the time loop (fdtd_grad).  Included by fdtd.cu (one
// translation unit: it launches the forward kernels for the recomputation).
//
// J = sum_n sum_p (Hz^{n+1/2}(p))^2.  Step n of the forward pass (fdtd.cu) is
//   H'  = H + chx (Ex_{j+1} - Ex_j) - chy (Ey_{i+1} - Ey_i)          (Eq. (5))
//   E'  = ca E + cb rd (dH') - cb J^n     on updated edges           (Eq. (3))
//   s'  = P s + Q h(H'),   E'(interface) = s'[:n_y]                  (Eq. (23))
// with the FP32 P, Q the forward uses.  Its transpose, backwards in n, with
// g = dJ/d(state after step n):
//   pre : g_s[:n_y] += g_E(interface); g_H'(h cells) += Q^T g_s; g_s <- P^T g_s;
//         g_H'(probes) += 2 o^n; dJ/dJ^n = -cb g_E on source edges;
//         half-cell material terms of the coupling (see below)
//   h   : g_H' += curl^T(cb g_E);  material gradients of the cell's edges
//   e   : g_E <- ca g_E (updated edges) + (H update)^T g_H'
// Edge materials are cell means, so a cell gets half of each edge's
//   dJ/deps_edge   = cb g_E (E^n - E^{n+1}) / dt,
//   dJ/dsigma_edge = -cb g_E (E^n + E^{n+1}) / 2.
// The coarse half cell of interface edge k enters the coupling of Eq. (19):
// with c_k = A1^{-1} e_k = Q[:, k] / (Dl G^T)_k and t = Q^T g_s,
//   dJ/deps_b,k   += (Dl Dl')_k / dt t_k / (Dl G^T)_k (y_k^n - y_k^{n+1})
//   dJ/dsigma_b,k -= (Dl Dl')_k / 2  t_k / (Dl G^T)_k (y_k^n + y_k^{n+1}).
// The forward pass is recomputed segment by segment from checkpoints; the E
// fields of a segment are kept as frames, Hz ping-pongs.

namespace {

struct AdjSimDev {
  float* gex[2];
  float* gey[2];
  float* ghz[2];
  const float* exF;    // E frames of the segment: frame t at exF + t * fstride
  const float* eyF;
  float* geps;         // FP32 per-cell accumulators of the segment (pitched)
  float* gsig;
  const float2* mat;
  long long fstride;
  int nx, ny, pitch, pad;
  float chx, chy, rdx, rdy;
  float inv_dt, pad2;
};

struct AdjInstDev {
  const float* M;        // [P | Q] FP32, n x ld (the forward's)
  float* gs[2];          // adjoint of [y; x~]
  const float* sF;       // state frames: frame t at sF + t * ld
  const int* y_edge;
  const int* h_cell;
  const float* lh_dt;    // (Dl Dl')_k / dt / (Dl G^T)_k
  const float* lh_2;     // (Dl Dl')_k / 2 / (Dl G^T)_k
  double* geps_b;        // per interface edge accumulators
  double* gsig_b;
  int n, ny, ld, sim;
};

struct AdjWork {         // one CTA of adj_pre: columns [c0, c1) of one instance
  int inst, c0, c1, pad;
};

struct AdjRun {
  const float* probe_out;   // [nsteps][nprobe] of the forward pass
  const float* seed;        // [nsteps][nprobe] dL/do^n (vector-Jacobian product), or null: 2 o^n (J)
  const int* probe_sim;
  const int* probe_cell;
  const SrcEdge* src_edges;
  float* dsrc;              // [nsrc][nsteps]
  long long nsteps;
  int nprobe, nedges;
};

__device__ __forceinline__ void cb_ca(float2 m1, float2 m2, float& ca, float& cb) {
  edge_coef(m1, m2, ca, cb);
}

// ROM transpose, probe and source terms of reverse step n (segment index t).
// A CTA of the model part takes kPreCols columns of one instance's [P | Q]
// and splits each column's sum over the rows into kPreSlices consecutive row
// slices, one warp each (in order r = r0, r0 + 1, ... within a slice, the
// loads of 16 rows in flight together); the slices' partial sums are added in
// slice order, so the result does not depend on scheduling.
constexpr int kPreCols = 32, kPreSlices = 8;

__global__ void __launch_bounds__(kPreCols * kPreSlices)
adj_pre_kernel(const AdjSimDev* __restrict__ sims, const AdjInstDev* __restrict__ insts,
               const AdjWork* __restrict__ work, int nwork, const AdjRun* __restrict__ ar,
               int par, int gpar, int t, long long n) {
  extern __shared__ float gsh[];   // g_s (n floats), then the slices' partial sums
  pdl_trigger();   // launched with programmatic serialisation: nothing read before pdl_wait
  pdl_wait();
  const int b = blockIdx.x;
  if (b < nwork) {
    const AdjWork w = work[b];
    const AdjInstDev ai = insts[w.inst];
    const AdjSimDev sd = sims[ai.sim];
    const float* __restrict__ gsa = gpar ? ai.gs[1] : ai.gs[0];
    float* __restrict__ gsb = gpar ? ai.gs[0] : ai.gs[1];
    const float* __restrict__ gexa = par ? sd.gex[1] : sd.gex[0];
    const float* __restrict__ geya = par ? sd.gey[1] : sd.gey[0];
    float* __restrict__ ghza = par ? sd.ghz[1] : sd.ghz[0];
    for (int k = threadIdx.x; k < ai.n; k += blockDim.x) {
      float g = gsa[k];
      if (k < ai.ny) {
        const int code = ai.y_edge[k];
        g += (code >> 30) ? geya[code & 0x3fffffff] : gexa[code & 0x3fffffff];
      }
      gsh[k] = g;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int c = w.c0 + lane;
    const int rps = (ai.n + kPreSlices - 1) / kPreSlices;
    const int r0 = sl * rps, r1 = min(ai.n, r0 + rps);
    float acc = 0.f;
    if (c < w.c1) {
      const float* __restrict__ Mc = ai.M + c;
      for (int rb = r0; rb < r1; rb += 16) {
        float mv[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) mv[u] = rb + u < r1 ? Mc[(size_t)(rb + u) * ai.ld] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (rb + u < r1) acc = fmaf(mv[u], gsh[rb + u], acc);
      }
    }
    float* part = gsh + ai.n;
    part[sl * kPreCols + lane] = acc;
    __syncthreads();
    if (sl == 0 && c < w.c1) {
      float tot = part[lane];
#pragma unroll
      for (int q = 1; q < kPreSlices; ++q) tot += part[q * kPreCols + lane];
      if (c < ai.n) {
        gsb[c] = tot;
      } else {
        const int k = c - ai.n;
        atomicAdd(ghza + ai.h_cell[k], tot);
        const float y0 = ai.sF[(size_t)t * ai.ld + k];
        const float y1 = ai.sF[(size_t)(t + 1) * ai.ld + k];
        ai.geps_b[k] += (double)ai.lh_dt[k] * tot * ((double)y0 - y1);
        ai.gsig_b[k] -= (double)ai.lh_2[k] * tot * ((double)y0 + y1);
      }
    }
    return;
  }
  const int idx = (b - nwork) * blockDim.x + threadIdx.x;
  if (idx < ar->nprobe) {
    const AdjSimDev* sd = sims + ar->probe_sim[idx];
    float* ghza = par ? sd->ghz[1] : sd->ghz[0];
    const size_t k = (size_t)n * ar->nprobe + idx;
    atomicAdd(ghza + ar->probe_cell[idx], ar->seed ? ar->seed[k] : 2.f * ar->probe_out[k]);
  } else if (idx - ar->nprobe < ar->nedges) {
    const SrcEdge se = ar->src_edges[idx - ar->nprobe];
    const AdjSimDev* sd = sims + se.sim;
    const size_t off = (size_t)se.j * sd->pitch + se.i;
    const float2 m2 = sd->mat[off];
    const float2 m1 = se.comp == 0 ? sd->mat[off - sd->pitch] : sd->mat[off - 1];
    float ca, cb;
    cb_ca(m1, m2, ca, cb);
    const float* ga = se.comp == 0 ? (par ? sd->gex[1] : sd->gex[0]) : (par ? sd->gey[1] : sd->gey[0]);
    atomicAdd(ar->dsrc + (size_t)se.src * ar->nsteps + n, -cb * ga[off]);
  }
}

// g_H' = g_H + curl^T(cb g_E) per coarse cell, and the cell's material terms.
__global__ void __launch_bounds__(256)
adj_h_kernel(const AdjSimDev* __restrict__ sims, const TileWork* __restrict__ tiles, int par, int t) {
  const TileWork tw = tiles[blockIdx.x];
  const AdjSimDev sd = sims[tw.sim];
  const int nx = sd.nx, ny = sd.ny, P = sd.pitch;
  const float* __restrict__ gex = par ? sd.gex[1] : sd.gex[0];
  const float* __restrict__ gey = par ? sd.gey[1] : sd.gey[0];
  const float* __restrict__ gha = par ? sd.ghz[1] : sd.ghz[0];
  float* __restrict__ ghb = par ? sd.ghz[0] : sd.ghz[1];
  const float* __restrict__ ex0 = sd.exF + (size_t)t * sd.fstride;
  const float* __restrict__ ex1 = ex0 + sd.fstride;
  const float* __restrict__ ey0 = sd.eyF + (size_t)t * sd.fstride;
  const float* __restrict__ ey1 = ey0 + sd.fstride;
  const float2* __restrict__ mat = sd.mat;
  const int w = min(kCtaCols, nx - tw.x0);
  for (int k = threadIdx.x; k < w * (tw.y1 - tw.y0); k += blockDim.x) {
    const int i = tw.x0 + k % w, j = tw.y0 + k / w;
    const size_t off = (size_t)j * P + i;
    const float2 m = mat[off];
    if (m.x < 0.f) {
      ghb[off] = 0.f;
      continue;
    }
    float g = gha[off], qe = 0.f, qs = 0.f, ca, cb;
    // Ex(i, j): cells (i, j-1), (i, j); Hz(i, j) enters with +cb rdy
    if (j >= 1) {
      const float2 mo = mat[off - P];
      if (mo.x >= 0.f) {
        cb_ca(mo, m, ca, cb);
        const float mu = cb * gex[off];
        g += sd.rdy * mu;
        qe += mu * (ex0[off] - ex1[off]);
        qs += mu * (ex0[off] + ex1[off]);
      }
    }
    // Ex(i, j+1): cells (i, j), (i, j+1); Hz(i, j) enters with -cb rdy
    if (j + 1 <= ny - 1) {
      const float2 mo = mat[off + P];
      if (mo.x >= 0.f) {
        cb_ca(m, mo, ca, cb);
        const float mu = cb * gex[off + P];
        g -= sd.rdy * mu;
        qe += mu * (ex0[off + P] - ex1[off + P]);
        qs += mu * (ex0[off + P] + ex1[off + P]);
      }
    }
    // Ey(i, j): cells (i-1, j), (i, j); Hz(i, j) enters with -cb rdx
    if (i >= 1) {
      const float2 mo = mat[off - 1];
      if (mo.x >= 0.f) {
        cb_ca(mo, m, ca, cb);
        const float mu = cb * gey[off];
        g -= sd.rdx * mu;
        qe += mu * (ey0[off] - ey1[off]);
        qs += mu * (ey0[off] + ey1[off]);
      }
    }
    // Ey(i+1, j): cells (i, j), (i+1, j); Hz(i, j) enters with +cb rdx
    if (i + 1 <= nx - 1) {
      const float2 mo = mat[off + 1];
      if (mo.x >= 0.f) {
        cb_ca(m, mo, ca, cb);
        const float mu = cb * gey[off + 1];
        g += sd.rdx * mu;
        qe += mu * (ey0[off + 1] - ey1[off + 1]);
        qs += mu * (ey0[off + 1] + ey1[off + 1]);
      }
    }
    ghb[off] = g;
    sd.geps[off] += 0.5f * sd.inv_dt * qe;   // times eps0 when flushed
    sd.gsig[off] -= 0.25f * qs;
  }
}

// g_E <- ca g_E (updated edges) + (H update)^T g_H' (updated and interface edges).
__global__ void __launch_bounds__(256)
adj_e_kernel(const AdjSimDev* __restrict__ sims, const TileWork* __restrict__ tiles, int par) {
  const TileWork tw = tiles[blockIdx.x];
  const AdjSimDev sd = sims[tw.sim];
  const int nx = sd.nx, P = sd.pitch;
  const float* __restrict__ gexa = par ? sd.gex[1] : sd.gex[0];
  const float* __restrict__ geya = par ? sd.gey[1] : sd.gey[0];
  float* __restrict__ gexb = par ? sd.gex[0] : sd.gex[1];
  float* __restrict__ geyb = par ? sd.gey[0] : sd.gey[1];
  const float* __restrict__ gh = par ? sd.ghz[0] : sd.ghz[1];   // g_H' just written
  const float2* __restrict__ mat = sd.mat;
  const int w = min(kCtaCols, nx - tw.x0);
  for (int k = threadIdx.x; k < w * (tw.y1 - tw.y0); k += blockDim.x) {
    const int i = tw.x0 + k % w, j = tw.y0 + k / w;
    const size_t off = (size_t)j * P + i;
    const float2 m = mat[off];
    float ca, cb;
    // Ex(i, j), 1 <= j <= ny-1: H(i, j-1) has +chx Ex, H(i, j) has -chx Ex
    float vx = 0.f;
    if (j >= 1) {
      const float2 mo = mat[off - P];
      const bool live_lo = mo.x >= 0.f, live_hi = m.x >= 0.f;
      if (live_lo || live_hi) {
        vx = sd.chx * ((live_lo ? gh[off - P] : 0.f) - (live_hi ? gh[off] : 0.f));
        if (live_lo && live_hi) {
          cb_ca(mo, m, ca, cb);
          vx += ca * gexa[off];
        }
      }
    }
    gexb[off] = vx;
    // Ey(i, j), 1 <= i <= nx-1: H(i, j) has +chy Ey, H(i-1, j) has -chy Ey
    float vy = 0.f;
    if (i >= 1) {
      const float2 mo = mat[off - 1];
      const bool live_l = mo.x >= 0.f, live_r = m.x >= 0.f;
      if (live_l || live_r) {
        vy = sd.chy * ((live_r ? gh[off] : 0.f) - (live_l ? gh[off - 1] : 0.f));
        if (live_l && live_r) {
          cb_ca(mo, m, ca, cb);
          vy += ca * geya[off];
        }
      }
    }
    geyb[off] = vy;
  }
}

// Fused form of adj_h + adj_e: one pass per reverse step, marching 128-column
// strips up the tile like the forward kernel (lane l owns 4 columns, float4
// loads, the next row's loads in flight while the current row is computed).
// Each E edge's mu = cb g_E and its material terms are formed once and used
// by both cells beside it; g_H'(j-1) is carried in registers for the Ex
// update of row j, g_H'(i-1) comes from the neighbouring lane (lane 0
// recomputes the halo column c0 - 1, the first row of a tile the halo row
// j0 - 1, neither of which accumulates material gradients).
struct AdjRowIn {
  float4 gx1, gy, gh;   // g_Ex(j+1), g_Ey(j), g_H(j) (after the model/probe terms)
  float4 m1a, m1b;      // mat(j+1)
  float4 x0, x1;        // Ex frames E^n, E^{n+1} of edge row j+1
  float4 y0, y1;        // Ey frames of row j
  float4 ae, as;        // the segment's eps / sigma accumulators of row j
  float gyR, y0R, y1R;  // lane 31: Ey edge (c0 + 128, j)
  float2 mR;            // lane 31: mat(c0 + 128, j)
  float gx1L, gyL, ghL; // lane 0: g_Ex(c0-1, j+1), g_Ey(c0-1, j), g_H(c0-1, j)
  float2 m1L, mLL;      // lane 0: mat(c0-1, j+1), mat(c0-2, j)
};

__device__ __forceinline__ void adj_load_row(AdjRowIn& r, const AdjSimDev& sd, const float* __restrict__ gexa,
                                             const float* __restrict__ geya, const float* __restrict__ gha,
                                             const float* __restrict__ ex0, const float* __restrict__ ex1,
                                             const float* __restrict__ ey0, const float* __restrict__ ey1,
                                             size_t row, int P, int cl, int c0, int lane, bool halo,
                                             bool right) {
  r.gx1 = ld4(gexa + row + P + cl);
  r.gy = ld4(geya + row + cl);
  r.gh = ld4(gha + row + cl);
  r.m1a = ld4(reinterpret_cast<const float*>(sd.mat + row + P + cl));
  r.m1b = ld4(reinterpret_cast<const float*>(sd.mat + row + P + cl + 2));
  r.x0 = ld4(ex0 + row + P + cl);
  r.x1 = ld4(ex1 + row + P + cl);
  r.y0 = ld4(ey0 + row + cl);
  r.y1 = ld4(ey1 + row + cl);
  r.ae = ld4(sd.geps + row + cl);
  r.as = ld4(sd.gsig + row + cl);
  if (right) {
    r.gyR = geya[row + c0 + 128];
    r.y0R = ey0[row + c0 + 128];
    r.y1R = ey1[row + c0 + 128];
    r.mR = sd.mat[row + c0 + 128];
  } else {
    r.gyR = r.y0R = r.y1R = 0.f;
    r.mR = make_float2(-1.f, 0.f);
  }
  if (halo) {
    r.gx1L = gexa[row + P + c0 - 1];
    r.gyL = geya[row + c0 - 1];
    r.ghL = gha[row + c0 - 1];
    r.m1L = sd.mat[row + P + c0 - 1];
    r.mLL = sd.mat[row + c0 - 2];
  } else {
    r.gx1L = r.gyL = r.ghL = 0.f;
    r.m1L = r.mLL = make_float2(-1.f, 0.f);
  }
}

// Staged form of the row loads (kRing >= 2): each lane copies its own eleven
// float4 of a row (and lanes 0 and 31 their halo scalars) into its warp's ring
// in shared memory with cp.async, kRing - 1 rows ahead of the row it computes,
// one commit group per row; the copies in flight hold no registers, so the
// kernel fits 128 registers (4 CTAs per SM) and keeps more bytes in flight.
// A lane reads back only what it copied itself.  Slot layout per warp:
// [11 values][32 lanes] float4, then 16 floats of halo scalars.
constexpr int kAdjSlot4 = 11 * 32 + 4;   // float4 per warp and ring slot

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

// The loads of adj_load_row, issued into a ring slot (then one commit group).
__device__ __forceinline__ void adj_issue_row(float4* slot, const AdjSimDev& sd, const float* __restrict__ gexa,
                                              const float* __restrict__ geya, const float* __restrict__ gha,
                                              const float* __restrict__ ex0, const float* __restrict__ ex1,
                                              const float* __restrict__ ey0, const float* __restrict__ ey1,
                                              size_t row, int P, int cl, int c0, int lane, bool halo, bool right) {
  asm volatile("" ::: "memory");   // after the reads of the slot's previous row
  cp_async16(slot + 0 * 32 + lane, gexa + row + P + cl, true);
  cp_async16(slot + 1 * 32 + lane, geya + row + cl, true);
  cp_async16(slot + 2 * 32 + lane, gha + row + cl, true);
  cp_async16(slot + 3 * 32 + lane, sd.mat + row + P + cl, true);
  cp_async16(slot + 4 * 32 + lane, sd.mat + row + P + cl + 2, true);
  cp_async16(slot + 5 * 32 + lane, ex0 + row + P + cl, true);
  cp_async16(slot + 6 * 32 + lane, ex1 + row + P + cl, true);
  cp_async16(slot + 7 * 32 + lane, ey0 + row + cl, true);
  cp_async16(slot + 8 * 32 + lane, ey1 + row + cl, true);
  cp_async16(slot + 9 * 32 + lane, sd.geps + row + cl, true);
  cp_async16(slot + 10 * 32 + lane, sd.gsig + row + cl, true);
  float* e = reinterpret_cast<float*>(slot + 11 * 32);
  if (halo) {
    cp_async4(e + 0, gexa + row + P + c0 - 1);
    cp_async4(e + 1, geya + row + c0 - 1);
    cp_async4(e + 2, gha + row + c0 - 1);
    cp_async8(e + 4, sd.mat + row + P + c0 - 1);
    cp_async8(e + 6, sd.mat + row + c0 - 2);
  }
  if (right) {
    cp_async4(e + 8, geya + row + c0 + 128);
    cp_async4(e + 9, ey0 + row + c0 + 128);
    cp_async4(e + 10, ey1 + row + c0 + 128);
    cp_async8(e + 12, sd.mat + row + c0 + 128);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void adj_fetch_row(AdjRowIn& r, const float4* slot, int lane, bool halo, bool right) {
  r.gx1 = slot[0 * 32 + lane];
  r.gy = slot[1 * 32 + lane];
  r.gh = slot[2 * 32 + lane];
  r.m1a = slot[3 * 32 + lane];
  r.m1b = slot[4 * 32 + lane];
  r.x0 = slot[5 * 32 + lane];
  r.x1 = slot[6 * 32 + lane];
  r.y0 = slot[7 * 32 + lane];
  r.y1 = slot[8 * 32 + lane];
  r.ae = slot[9 * 32 + lane];
  r.as = slot[10 * 32 + lane];
  const float* e = reinterpret_cast<const float*>(slot + 11 * 32);
  if (right) {
    r.gyR = e[8];
    r.y0R = e[9];
    r.y1R = e[10];
    r.mR = make_float2(e[12], e[13]);
  } else {
    r.gyR = r.y0R = r.y1R = 0.f;
    r.mR = make_float2(-1.f, 0.f);
  }
  if (halo) {
    r.gx1L = e[0];
    r.gyL = e[1];
    r.ghL = e[2];
    r.m1L = make_float2(e[4], e[5]);
    r.mLL = make_float2(e[6], e[7]);
  } else {
    r.gx1L = r.gyL = r.ghL = 0.f;
    r.m1L = r.mLL = make_float2(-1.f, 0.f);
  }
}

template <int kRing, int kMinBlocks>
__global__ void __launch_bounds__(128, kMinBlocks)
adj_cell_kernel(const AdjSimDev* __restrict__ sims, const TileWork* __restrict__ tiles, int par, int t) {
  extern __shared__ float4 adj_ring[];
  pdl_trigger();   // launched with programmatic serialisation: nothing read before pdl_wait
  pdl_wait();
  const unsigned FULL = 0xffffffffu;
  const TileWork tw = tiles[blockIdx.x];
  const AdjSimDev sd = sims[tw.sim];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = tw.x0 + warp * 128;
  const int nx = sd.nx, ny = sd.ny, P = sd.pitch;
  if (c0 >= nx) return;
  const float* __restrict__ gexa = par ? sd.gex[1] : sd.gex[0];
  const float* __restrict__ geya = par ? sd.gey[1] : sd.gey[0];
  const float* __restrict__ gha = par ? sd.ghz[1] : sd.ghz[0];
  float* __restrict__ gexb = par ? sd.gex[0] : sd.gex[1];
  float* __restrict__ geyb = par ? sd.gey[0] : sd.gey[1];
  float* __restrict__ ghb = par ? sd.ghz[0] : sd.ghz[1];
  const float* __restrict__ ex0 = sd.exF + (size_t)t * sd.fstride;
  const float* __restrict__ ex1 = ex0 + sd.fstride;
  const float* __restrict__ ey0 = sd.eyF + (size_t)t * sd.fstride;
  const float* __restrict__ ey1 = ey0 + sd.fstride;
  const int cl = c0 + 4 * lane;
  const int j0 = tw.y0, j1 = tw.y1;
  const int js = j0 > 0 ? j0 - 1 : 0;
  const bool halo = lane == 0 && c0 > 0;
  const bool right = lane == 31 && c0 + 128 <= nx - 1;
  // carried state: mat(j), mu / material terms / ca of the Ex edges of row j
  // (cells j-1, j), g_Ex(j), g_H'(j-1); lane 0 the same for column c0 - 1
  float2 mj[4];
  float mux[4], edx[4], esx[4], cgx[4], ghp[4];   // cgx = ca g_Ex of the Ex edges of row j
  float2 mjL = make_float2(-1.f, 0.f);
  float muxL = 0.f;
  {
    const size_t row = (size_t)js * P;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mj[q] = sd.mat[row + cl + q];
      mux[q] = edx[q] = esx[q] = cgx[q] = ghp[q] = 0.f;
      if (js >= 1 && cl + q < nx) {
        const float2 mo = sd.mat[row - P + cl + q];
        if (mo.x >= 0.f && mj[q].x >= 0.f) {
          float ca, cb;
          cb_ca(mo, mj[q], ca, cb);
          mux[q] = cb * gexa[row + cl + q];
        }
      }
    }
    if (halo) {
      mjL = sd.mat[row + c0 - 1];
      if (js >= 1) {
        const float2 mo = sd.mat[row - P + c0 - 1];
        if (mo.x >= 0.f && mjL.x >= 0.f) {
          float ca, cb;
          cb_ca(mo, mjL, ca, cb);
          muxL = cb * gexa[row + c0 - 1];
        }
      }
    }
  }
  AdjRowIn cur, nxt;
  float4* ring = adj_ring + (size_t)warp * (kRing > 0 ? kRing : 1) * kAdjSlot4;
  int slot = 0;
  if constexpr (kRing > 0) {
#pragma unroll
    for (int d = 0; d < kRing - 1; ++d) {
      if (js + d < j1)
        adj_issue_row(ring + d * kAdjSlot4, sd, gexa, geya, gha, ex0, ex1, ey0, ey1, (size_t)(js + d) * P, P, cl, c0,
                      lane, halo, right);
      else
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
  } else {
    adj_load_row(cur, sd, gexa, geya, gha, ex0, ex1, ey0, ey1, (size_t)js * P, P, cl, c0, lane, halo, right);
  }
  for (int j = js; j < j1; ++j) {
    const size_t row = (size_t)j * P;
    if constexpr (kRing > 0) {
      int ahead = slot + kRing - 1;
      ahead -= ahead >= kRing ? kRing : 0;
      // row j + kRing - 1 (past the tile: an empty group, so the count stays uniform)
      if (j + kRing - 1 < j1)
        adj_issue_row(ring + ahead * kAdjSlot4, sd, gexa, geya, gha, ex0, ex1, ey0, ey1, row + (size_t)(kRing - 1) * P,
                      P, cl, c0, lane, halo, right);
      else
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      cp_async_wait_n<kRing - 1>();
      adj_fetch_row(cur, ring + slot * kAdjSlot4, lane, halo, right);
      slot = slot + 1 == kRing ? 0 : slot + 1;
    } else {
      if (j + 1 < j1)
        adj_load_row(nxt, sd, gexa, geya, gha, ex0, ex1, ey0, ey1, row + P, P, cl, c0, lane, halo, right);
    }
    const float2 m1[4] = {make_float2(cur.m1a.x, cur.m1a.y), make_float2(cur.m1a.z, cur.m1a.w),
                          make_float2(cur.m1b.x, cur.m1b.y), make_float2(cur.m1b.z, cur.m1b.w)};
    // Ex edges of row j+1 (cells j, j+1)
    float mux1[4], edx1[4], esx1[4], cgx1[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mux1[q] = edx1[q] = esx1[q] = cgx1[q] = 0.f;
      if (j + 1 <= ny - 1 && cl + q < nx && mj[q].x >= 0.f && m1[q].x >= 0.f) {
        float ca, cb;
        cb_ca(mj[q], m1[q], ca, cb);
        const float mu = cb * comp(cur.gx1, q);
        mux1[q] = mu;
        edx1[q] = mu * (comp(cur.x0, q) - comp(cur.x1, q));
        esx1[q] = mu * (comp(cur.x0, q) + comp(cur.x1, q));
        cgx1[q] = ca * comp(cur.gx1, q);
      }
    }
    // Ey edges of row j at i = cl + q (cells i-1, i)
    float2 mleft = make_float2(__shfl_up_sync(FULL, mj[3].x, 1), __shfl_up_sync(FULL, mj[3].y, 1));
    if (lane == 0) mleft = mjL;
    float muy[4], edy[4], esy[4], cay[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = cl + q;
      const float2 ml = q == 0 ? mleft : mj[q - 1];
      muy[q] = edy[q] = esy[q] = cay[q] = 0.f;
      if (i >= 1 && i <= nx - 1 && ml.x >= 0.f && mj[q].x >= 0.f) {
        float ca, cb;
        cb_ca(ml, mj[q], ca, cb);
        const float mu = cb * comp(cur.gy, q);
        muy[q] = mu;
        edy[q] = mu * (comp(cur.y0, q) - comp(cur.y1, q));
        esy[q] = mu * (comp(cur.y0, q) + comp(cur.y1, q));
        cay[q] = ca;
      }
    }
    // the Ey edge right of the lane's last column: the next lane's first
    float muyR = __shfl_down_sync(FULL, muy[0], 1);
    float edyR = __shfl_down_sync(FULL, edy[0], 1);
    float esyR = __shfl_down_sync(FULL, esy[0], 1);
    if (lane == 31) {
      muyR = edyR = esyR = 0.f;
      if (right && mj[3].x >= 0.f && cur.mR.x >= 0.f) {
        float ca, cb;
        cb_ca(mj[3], cur.mR, ca, cb);
        muyR = cb * cur.gyR;
        edyR = muyR * (cur.y0R - cur.y1R);
        esyR = muyR * (cur.y0R + cur.y1R);
      }
    }
    // g_H' of the row's cells and their material terms
    // (the accumulators were loaded with the row; cells that take no term
    // keep their value, and only the tile's own rows are written back)
    float gn[4], ae[4], as[4];
    const bool own = j >= j0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool live = cl + q < nx && mj[q].x >= 0.f;
      const float mr = q < 3 ? muy[q + 1] : muyR;
      gn[q] = live ? comp(cur.gh, q) + sd.rdy * mux[q] - sd.rdy * mux1[q] - sd.rdx * muy[q] + sd.rdx * mr : 0.f;
      ae[q] = comp(cur.ae, q);
      as[q] = comp(cur.as, q);
      if (live) {
        const float er = q < 3 ? edy[q + 1] : edyR;
        const float sr = q < 3 ? esy[q + 1] : esyR;
        const float qe = edx[q] + edx1[q] + edy[q] + er;
        const float qs = esx[q] + esx1[q] + esy[q] + sr;
        ae[q] += 0.5f * sd.inv_dt * qe;
        as[q] -= 0.25f * qs;
      }
    }
    if (own) {
      st4(sd.geps + row + cl, make_float4(ae[0], ae[1], ae[2], ae[3]));
      st4(sd.gsig + row + cl, make_float4(as[0], as[1], as[2], as[3]));
    }
    // lane 0: g_H' of the halo column c0 - 1
    float gnL = 0.f;
    if (halo) {
      float muxL1 = 0.f, muyL = 0.f;
      float ca, cb;
      if (j + 1 <= ny - 1 && mjL.x >= 0.f && cur.m1L.x >= 0.f) {
        cb_ca(mjL, cur.m1L, ca, cb);
        muxL1 = cb * cur.gx1L;
      }
      if (c0 - 1 >= 1 && cur.mLL.x >= 0.f && mjL.x >= 0.f) {
        cb_ca(cur.mLL, mjL, ca, cb);
        muyL = cb * cur.gyL;
      }
      gnL = mjL.x >= 0.f ? cur.ghL + sd.rdy * muxL - sd.rdy * muxL1 - sd.rdx * muyL + sd.rdx * muy[0] : 0.f;
      muxL = muxL1;
    }
    float gL = __shfl_up_sync(FULL, gn[3], 1);
    if (lane == 0) gL = gnL;
    if (own) {
      float vx[4], vy[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = cl + q;
        // Ex(i, j): H(i, j-1) has +chx Ex, H(i, j) has -chx Ex (g_H' = 0 on covered cells)
        float v = 0.f;
        if (j >= 1 && i < nx) {
          v = sd.chx * (ghp[q] - gn[q]);
          v += cgx[q];   // 0 unless both cells are coarse cells
        }
        vx[q] = v;
        // Ey(i, j): H(i, j) has +chy Ey, H(i-1, j) has -chy Ey
        float w = 0.f;
        if (i >= 1 && i < nx) {
          w = sd.chy * (gn[q] - (q == 0 ? gL : gn[q - 1]));
          w += cay[q] * comp(cur.gy, q);
        }
        vy[q] = w;
      }
      st4(gexb + row + cl, make_float4(vx[0], vx[1], vx[2], vx[3]));
      st4(geyb + row + cl, make_float4(vy[0], vy[1], vy[2], vy[3]));
      st4(ghb + row + cl, make_float4(gn[0], gn[1], gn[2], gn[3]));
    }
    // carry to row j + 1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mj[q] = m1[q];
      mux[q] = mux1[q];
      edx[q] = edx1[q];
      esx[q] = esx1[q];
      cgx[q] = cgx1[q];
      ghp[q] = gn[q];
    }
    if (halo) mjL = cur.m1L;
    if constexpr (kRing == 0) cur = nxt;
  }
}

// ---------------------------------------------------------------------------
// Two reverse steps per pass (row marching, like the forward's
// yee_tb2m_kernel).  Iteration j runs
//   A: reverse step t at row j (adj_cell_kernel's arithmetic: g_H' of the
//      row's cells from g_E of rows j and j + 1, then g_E' of row j), and
//   B: reverse step t - 1 at row j - 1, from A's rows j - 1 and j,
// holding A's results in registers, and stores B's row (and the accumulators
// of both steps) when the tile owns it.  A and B start two rows below the
// tile (their first row's carried edge terms are not known, which reaches
// only rows that are not stored).  The additions that precede reverse step
// t - 1 (the transposed maps' Q^T g_s on the cells beside each model, the
// probe seeds) are left out here and made afterwards by adj_fix_kernel: the
// reverse step is linear in (g_E, g_H) for fixed frames, and adding d to
// g_H of a cell before it adds d to that cell's g_H' and -chx d, +chx d,
// +chy d, -chy d to the g_E' of its lower, upper, left and right edges, and
// nothing else (the material terms read g_E and the frames only).  A exports
// its g_E of the edges those additions read (interface and source edges).
// A warp computes the 128 columns [c0 - 4, c0 + 124) and stores
// [c0, c0 + 120): lane l holds c0 - 4 + 4 l .. + 3 and neighbour values come
// from shuffles (wrong in the outer columns, which nothing stored reads).
// A CTA has W = 3 or 4 warps (blockDim.x / 32) and covers W x 120 columns:
// W is chosen per run so that the grids' last column blocks leave the
// fewest warps idle (1024 columns: three CTAs of three warps, no idle warp).
// The row loads are staged one row ahead through shared memory (cp.async).

struct AdjExp {     // an edge whose g_E after reverse step t is exported
  int j, i, comp, slot;
};

struct AdjMarchDev {
  const int2* exp_rng;   // per warp (tile * W + warp): [begin, end) into exp, rows ascending
  const AdjExp* exp;
  float* expv;           // the exported values, by slot
};

constexpr int kAdj2Vals = 13;               // float4 per lane and row in the ring
constexpr int kAdj2Slot4 = kAdj2Vals * 32;  // per warp and ring slot
constexpr size_t kAdj2SmemPerWarp = (size_t)2 * kAdj2Slot4 * sizeof(float4);

// Row j's loads: g_Ex(j + 1), g_Ey(j), g_H(j), mat(j + 1), the Ex frames of
// edge row j + 1 and the Ey frames of row j at t - 1, t, t + 1, and the
// accumulators of row j (one commit group).
__device__ __forceinline__ void adj2_issue(float4* slot, const AdjSimDev& sd, const float* gexa, const float* geya,
                                           const float* gha, const float* xm, const float* y_m, size_t fs,
                                           size_t row, int P, int cl, int lane, bool ok) {
  asm volatile("" ::: "memory");   // after the reads of the slot's previous row
  const size_t r0 = ok ? row + cl : 0, r1 = ok ? row + P + cl : 0;
  cp_async16(slot + 0 * 32 + lane, gexa + r1, ok);
  cp_async16(slot + 1 * 32 + lane, geya + r0, ok);
  cp_async16(slot + 2 * 32 + lane, gha + r0, ok);
  cp_async16(slot + 3 * 32 + lane, sd.mat + r1, ok);
  cp_async16(slot + 4 * 32 + lane, sd.mat + r1 + 2, ok);
  cp_async16(slot + 5 * 32 + lane, xm + r1, ok);
  cp_async16(slot + 6 * 32 + lane, xm + fs + r1, ok);
  cp_async16(slot + 7 * 32 + lane, xm + 2 * fs + r1, ok);
  cp_async16(slot + 8 * 32 + lane, y_m + r0, ok);
  cp_async16(slot + 9 * 32 + lane, y_m + fs + r0, ok);
  cp_async16(slot + 10 * 32 + lane, y_m + 2 * fs + r0, ok);
  cp_async16(slot + 11 * 32 + lane, sd.geps + r0, ok);
  cp_async16(slot + 12 * 32 + lane, sd.gsig + r0, ok);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// One reverse step at row j (adj_cell_kernel's operations in its order):
// from the row's inputs and the carried terms of the Ex edges of row j
// (mux, edx, esx, cgx) and g_H'(j - 1) (ghp), the row's g_H' (gn), g_E' of
// its Ex and Ey edges (vx, vy) and its cells' material terms (qe, qs, taken
// where live); the carried terms move on to the Ex edges of row j + 1.
__device__ __forceinline__ void adj2_row(const AdjSimDev& sd, int j, int cl, const float2 (&mj)[4],
                                         const float2 (&m1)[4], const float4& gx1, const float4& gy, const float4& gh,
                                         const float4& x0, const float4& x1, const float4& y0, const float4& y1,
                                         float (&mux)[4], float (&edx)[4], float (&esx)[4], float (&cgx)[4],
                                         const float (&ghp)[4], float (&gn)[4], float (&vx)[4], float (&vy)[4],
                                         float (&qe)[4], float (&qs)[4], bool (&live)[4]) {
  const unsigned FULL = 0xffffffffu;
  const int nx = sd.nx, ny = sd.ny;
  float mux1[4], edx1[4], esx1[4], cgx1[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    mux1[q] = edx1[q] = esx1[q] = cgx1[q] = 0.f;
    if (j + 1 <= ny - 1 && cl + q < nx && mj[q].x >= 0.f && m1[q].x >= 0.f) {
      float ca, cb;
      cb_ca(mj[q], m1[q], ca, cb);
      const float mu = cb * comp(gx1, q);
      mux1[q] = mu;
      edx1[q] = mu * (comp(x0, q) - comp(x1, q));
      esx1[q] = mu * (comp(x0, q) + comp(x1, q));
      cgx1[q] = ca * comp(gx1, q);
    }
  }
  const float2 mleft = make_float2(__shfl_up_sync(FULL, mj[3].x, 1), __shfl_up_sync(FULL, mj[3].y, 1));
  float muy[4], edy[4], esy[4], cay[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = cl + q;
    const float2 ml = q == 0 ? mleft : mj[q - 1];
    muy[q] = edy[q] = esy[q] = cay[q] = 0.f;
    if (i >= 1 && i <= nx - 1 && ml.x >= 0.f && mj[q].x >= 0.f) {
      float ca, cb;
      cb_ca(ml, mj[q], ca, cb);
      const float mu = cb * comp(gy, q);
      muy[q] = mu;
      edy[q] = mu * (comp(y0, q) - comp(y1, q));
      esy[q] = mu * (comp(y0, q) + comp(y1, q));
      cay[q] = ca;
    }
  }
  const float muyR = __shfl_down_sync(FULL, muy[0], 1);
  const float edyR = __shfl_down_sync(FULL, edy[0], 1);
  const float esyR = __shfl_down_sync(FULL, esy[0], 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    live[q] = cl + q < nx && mj[q].x >= 0.f;
    const float mr = q < 3 ? muy[q + 1] : muyR;
    gn[q] = live[q] ? comp(gh, q) + sd.rdy * mux[q] - sd.rdy * mux1[q] - sd.rdx * muy[q] + sd.rdx * mr : 0.f;
    const float er = q < 3 ? edy[q + 1] : edyR;
    const float sr = q < 3 ? esy[q + 1] : esyR;
    qe[q] = edx[q] + edx1[q] + edy[q] + er;
    qs[q] = esx[q] + esx1[q] + esy[q] + sr;
  }
  const float gL = __shfl_up_sync(FULL, gn[3], 1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = cl + q;
    float v = 0.f;
    if (j >= 1 && i < nx) {
      v = sd.chx * (ghp[q] - gn[q]);
      v += cgx[q];
    }
    vx[q] = v;
    float w = 0.f;
    if (i >= 1 && i < nx) {
      w = sd.chy * (gn[q] - (q == 0 ? gL : gn[q - 1]));
      w += cay[q] * comp(gy, q);
    }
    vy[q] = w;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    mux[q] = mux1[q];
    edx[q] = edx1[q];
    esx[q] = esx1[q];
    cgx[q] = cgx1[q];
  }
}

__device__ __forceinline__ float adj2_pick(const float (&v)[4], int t) {
  return t == 0 ? v[0] : (t == 1 ? v[1] : (t == 2 ? v[2] : v[3]));
}

__global__ void __launch_bounds__(128, 3)
adj_march_kernel(const AdjSimDev* __restrict__ sims, const TileWork* __restrict__ tiles,
                 const AdjMarchDev* __restrict__ am, int par, int t) {
  extern __shared__ float4 adj2_ring[];
  pdl_trigger();   // launched with programmatic serialisation: nothing read before pdl_wait
  pdl_wait();
  const TileWork tw = tiles[blockIdx.x];
  const AdjSimDev sd = sims[tw.sim];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = tw.x0 + kMarchOut * warp;
  const int nx = sd.nx, ny = sd.ny, P = sd.pitch;
  if (c0 >= nx) return;
  const int wi = blockIdx.x * (blockDim.x >> 5) + warp;
  const float* __restrict__ gexa = par ? sd.gex[1] : sd.gex[0];
  const float* __restrict__ geya = par ? sd.gey[1] : sd.gey[0];
  const float* __restrict__ gha = par ? sd.ghz[1] : sd.ghz[0];
  float* __restrict__ gexb = par ? sd.gex[0] : sd.gex[1];
  float* __restrict__ geyb = par ? sd.gey[0] : sd.gey[1];
  float* __restrict__ ghb = par ? sd.ghz[0] : sd.ghz[1];
  const size_t fs = (size_t)sd.fstride;
  const float* xm = sd.exF + (size_t)(t - 1) * fs;   // frames t - 1, t, t + 1 at xm, xm + fs, xm + 2 fs
  const float* y_m = sd.eyF + (size_t)(t - 1) * fs;
  const int cl = c0 - 4 + 4 * lane;
  const bool inb = cl >= 0 && cl < P;
  const bool owner = lane >= 1 && lane <= 30 && cl < nx;
  const int j0 = tw.y0, j1 = tw.y1;
  const int jA0 = j0 >= 2 ? j0 - 2 : 0;       // A's and B's first row
  const int jAe = j1 < ny ? j1 : ny - 1;      // A's last row (row ny: the boundary's Ex edges, zero)
  const int2 er = am->exp_rng[wi];
  int ke = er.x;
  AdjExp ea = ke < er.y ? am->exp[ke] : AdjExp{kMarchNone, 0, 0, 0};
  const float2 dead = make_float2(-1.f, 0.f);
  // A's carried state at its first row: mat(jA0), the Ex edges of row jA0
  float2 mj[4];
  float muxA[4], edxA[4], esxA[4], cgxA[4], ghpA[4];
  {
    const size_t row = (size_t)jA0 * P;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mj[q] = inb ? sd.mat[row + cl + q] : dead;
      muxA[q] = edxA[q] = esxA[q] = cgxA[q] = ghpA[q] = 0.f;
      if (inb && jA0 >= 1 && cl + q < nx) {
        const float2 mo = sd.mat[row - P + cl + q];
        if (mo.x >= 0.f && mj[q].x >= 0.f) {
          float ca, cb;
          cb_ca(mo, mj[q], ca, cb);
          muxA[q] = cb * gexa[row + cl + q];
        }
      }
    }
  }
  // B's carried state (its first row's Ex-edge terms start at zero) and what
  // it takes from A's previous row: mat, g_Ey', the frames, the accumulators
  float2 mP[4];
  float muxB[4], edxB[4], esxB[4], cgxB[4], ghpB[4], vyP[4], aeP[4], asP[4];
  float4 xbm = make_float4(0.f, 0.f, 0.f, 0.f), xb0 = xbm, ybm = xbm, yb0 = xbm;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    mP[q] = dead;
    muxB[q] = edxB[q] = esxB[q] = cgxB[q] = ghpB[q] = vyP[q] = aeP[q] = asP[q] = 0.f;
  }
  float4* ring = adj2_ring + (size_t)warp * 2 * kAdj2Slot4;
  adj2_issue(ring, sd, gexa, geya, gha, xm, y_m, fs, (size_t)jA0 * P, P, cl, lane, inb);
  int slot = 0;
  for (int j = jA0; j <= j1; ++j) {
    if (j + 1 <= jAe)
      adj2_issue(ring + (slot ^ 1) * kAdj2Slot4, sd, gexa, geya, gha, xm, y_m, fs, (size_t)(j + 1) * P, P, cl, lane,
                 inb);
    else
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    cp_async_wait_n<1>();
    const float4* cs = ring + slot * kAdj2Slot4;
    slot ^= 1;
    // ---- A: reverse step t at row j
    float gnA[4], vxA[4], vyA[4], aeA[4], asA[4];
    float2 m1[4];
    float4 xfm = make_float4(0.f, 0.f, 0.f, 0.f), xf0 = xfm, yfm = xfm, yf0 = xfm;
    if (j <= jAe) {
      const float4 gx1 = cs[0 * 32 + lane], gy = cs[1 * 32 + lane], gh = cs[2 * 32 + lane];
      const float4 ma = cs[3 * 32 + lane], mb = cs[4 * 32 + lane];
      m1[0] = make_float2(ma.x, ma.y), m1[1] = make_float2(ma.z, ma.w);
      m1[2] = make_float2(mb.x, mb.y), m1[3] = make_float2(mb.z, mb.w);
      if (!inb) m1[0] = m1[1] = m1[2] = m1[3] = dead;
      xfm = cs[5 * 32 + lane], xf0 = cs[6 * 32 + lane];
      const float4 xfp = cs[7 * 32 + lane];
      yfm = cs[8 * 32 + lane], yf0 = cs[9 * 32 + lane];
      const float4 yfp = cs[10 * 32 + lane];
      const float4 ae4 = cs[11 * 32 + lane], as4 = cs[12 * 32 + lane];
      float qe[4], qs[4];
      bool live[4];
      adj2_row(sd, j, cl, mj, m1, gx1, gy, gh, xf0, xfp, yf0, yfp, muxA, edxA, esxA, cgxA, ghpA, gnA, vxA, vyA, qe,
               qs, live);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        aeA[q] = comp(ae4, q);
        asA[q] = comp(as4, q);
        if (live[q]) {
          aeA[q] += 0.5f * sd.inv_dt * qe[q];
          asA[q] -= 0.25f * qs[q];
        }
      }
      // the exported edges of this row (owned rows only, in the lists)
      while (ea.j == j) {
        const int q = ea.i - cl;
        if (owner && q >= 0 && q < 4) am->expv[ea.slot] = adj2_pick(ea.comp == 0 ? vxA : vyA, q);
        ++ke;
        ea = ke < er.y ? am->exp[ke] : AdjExp{kMarchNone, 0, 0, 0};
      }
    } else {   // j = ny: only B's last row remains
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        gnA[q] = vxA[q] = vyA[q] = aeA[q] = asA[q] = 0.f;
        m1[q] = dead;
      }
    }
    // ---- B: reverse step t - 1 at row r = j - 1
    const int r = j - 1;
    if (r >= jA0) {
      const float4 gx1 = make_float4(vxA[0], vxA[1], vxA[2], vxA[3]);
      const float4 gy = make_float4(vyP[0], vyP[1], vyP[2], vyP[3]);
      const float4 gh = make_float4(ghpA[0], ghpA[1], ghpA[2], ghpA[3]);
      float gnB[4], vxB[4], vyB[4], qe[4], qs[4];
      bool live[4];
      adj2_row(sd, r, cl, mP, mj, gx1, gy, gh, xbm, xb0, ybm, yb0, muxB, edxB, esxB, cgxB, ghpB, gnB, vxB, vyB, qe,
               qs, live);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (live[q]) {
          aeP[q] += 0.5f * sd.inv_dt * qe[q];
          asP[q] -= 0.25f * qs[q];
        }
      if (owner && r >= j0) {
        const size_t off = (size_t)r * P + cl;
        st4(gexb + off, make_float4(vxB[0], vxB[1], vxB[2], vxB[3]));
        st4(geyb + off, make_float4(vyB[0], vyB[1], vyB[2], vyB[3]));
        st4(ghb + off, make_float4(gnB[0], gnB[1], gnB[2], gnB[3]));
        st4(sd.geps + off, make_float4(aeP[0], aeP[1], aeP[2], aeP[3]));
        st4(sd.gsig + off, make_float4(asP[0], asP[1], asP[2], asP[3]));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) ghpB[q] = gnB[q];
    }
    // ---- carry to row j + 1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mP[q] = mj[q];
      mj[q] = m1[q];
      ghpA[q] = gnA[q];
      vyP[q] = vyA[q];
      aeP[q] = aeA[q];
      asP[q] = asA[q];
    }
    xbm = xfm, xb0 = xf0, ybm = yfm, yb0 = yf0;
  }
}

// After adj_march_kernel: the additions that precede reverse step n (the
// second step of the pass, segment index t): the transposed maps with the
// exported g_E of the interface edges (adj_pre_kernel's model part, into the
// other g_s buffer; its Q^T g_s on the cells beside the model), the probe
// seeds and the source gradients; each addition d to g_H of a live cell is
// applied to the pass's output as the cell pass would have carried it (the
// cell's g_H' and its four edges' g_E').
__device__ __forceinline__ void adj_fix_cell(const AdjSimDev& sd, float* gexb, float* geyb, float* ghb, int cell,
                                             float d) {
  const int P = sd.pitch, i = cell % P, j = cell / P;
  if (sd.mat[cell].x < 0.f) return;   // the cell pass leaves covered cells at zero
  atomicAdd(ghb + cell, d);
  if (j >= 1) atomicAdd(gexb + cell, -(sd.chx * d));
  if (j + 1 <= sd.ny - 1) atomicAdd(gexb + cell + P, sd.chx * d);
  if (i >= 1) atomicAdd(geyb + cell, sd.chy * d);
  if (i + 1 <= sd.nx - 1) atomicAdd(geyb + cell + 1, -(sd.chy * d));
}

__global__ void __launch_bounds__(kPreCols * kPreSlices)
adj_fix_kernel(const AdjSimDev* __restrict__ sims, const AdjInstDev* __restrict__ insts,
               const AdjWork* __restrict__ work, int nwork, const AdjRun* __restrict__ ar,
               const float* __restrict__ expv, const int* __restrict__ inst_exp, int src_exp, int bpar, int gpar,
               int t, long long n) {
  extern __shared__ float gsh[];   // g_s (n floats), then the slices' partial sums
  pdl_trigger();
  pdl_wait();
  const int b = blockIdx.x;
  if (b < nwork) {
    const AdjWork w = work[b];
    const AdjInstDev ai = insts[w.inst];
    const AdjSimDev sd = sims[ai.sim];
    const float* __restrict__ gsa = gpar ? ai.gs[1] : ai.gs[0];
    float* __restrict__ gsb = gpar ? ai.gs[0] : ai.gs[1];
    float* __restrict__ gexb = bpar ? sd.gex[1] : sd.gex[0];
    float* __restrict__ geyb = bpar ? sd.gey[1] : sd.gey[0];
    float* __restrict__ ghb = bpar ? sd.ghz[1] : sd.ghz[0];
    const float* __restrict__ ev = expv + inst_exp[w.inst];
    for (int k = threadIdx.x; k < ai.n; k += blockDim.x) {
      float g = gsa[k];
      if (k < ai.ny) g += ev[k];
      gsh[k] = g;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int c = w.c0 + lane;
    const int rps = (ai.n + kPreSlices - 1) / kPreSlices;
    const int r0 = sl * rps, r1 = min(ai.n, r0 + rps);
    float acc = 0.f;
    if (c < w.c1) {
      const float* __restrict__ Mc = ai.M + c;
      for (int rb = r0; rb < r1; rb += 16) {
        float mv[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) mv[u] = rb + u < r1 ? Mc[(size_t)(rb + u) * ai.ld] : 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (rb + u < r1) acc = fmaf(mv[u], gsh[rb + u], acc);
      }
    }
    float* part = gsh + ai.n;
    part[sl * kPreCols + lane] = acc;
    __syncthreads();
    if (sl == 0 && c < w.c1) {
      float tot = part[lane];
#pragma unroll
      for (int q = 1; q < kPreSlices; ++q) tot += part[q * kPreCols + lane];
      if (c < ai.n) {
        gsb[c] = tot;
      } else {
        const int k = c - ai.n;
        adj_fix_cell(sd, gexb, geyb, ghb, ai.h_cell[k], tot);
        const float y0 = ai.sF[(size_t)t * ai.ld + k];
        const float y1 = ai.sF[(size_t)(t + 1) * ai.ld + k];
        ai.geps_b[k] += (double)ai.lh_dt[k] * tot * ((double)y0 - y1);
        ai.gsig_b[k] -= (double)ai.lh_2[k] * tot * ((double)y0 + y1);
      }
    }
    return;
  }
  const int idx = (b - nwork) * blockDim.x + threadIdx.x;
  if (idx < ar->nprobe) {
    const AdjSimDev* sd = sims + ar->probe_sim[idx];
    const size_t k = (size_t)n * ar->nprobe + idx;
    adj_fix_cell(*sd, bpar ? sd->gex[1] : sd->gex[0], bpar ? sd->gey[1] : sd->gey[0], bpar ? sd->ghz[1] : sd->ghz[0],
                 ar->probe_cell[idx], ar->seed ? ar->seed[k] : 2.f * ar->probe_out[k]);
  } else if (idx - ar->nprobe < ar->nedges) {
    const int e = idx - ar->nprobe;
    const SrcEdge se = ar->src_edges[e];
    const AdjSimDev* sd = sims + se.sim;
    const size_t off = (size_t)se.j * sd->pitch + se.i;
    const float2 m2 = sd->mat[off];
    const float2 m1 = se.comp == 0 ? sd->mat[off - sd->pitch] : sd->mat[off - 1];
    float ca, cb;
    cb_ca(m1, m2, ca, cb);
    atomicAdd(ar->dsrc + (size_t)se.src * ar->nsteps + n, -cb * expv[src_exp + e]);
  }
}

// Moves a segment's FP32 accumulators into the FP64 totals and clears them.
__global__ void adj_flush_kernel(float* __restrict__ g32, double* __restrict__ g64, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    g64[k] += g32[k];
    g32[k] = 0.f;
  }
}

// Dense per-simulation outputs from the pitched FP64 totals.
__global__ void adj_out_kernel(const double* __restrict__ ge, const double* __restrict__ gs, int nx,
                               int ny, int pitch, const float2* __restrict__ mat, float* __restrict__ oe,
                               float* __restrict__ os) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nx * ny; k += gridDim.x * blockDim.x) {
    const int i = k % nx, j = k / nx;
    const size_t off = (size_t)j * pitch + i;
    const bool live = mat[off].x >= 0.f;
    if (oe) oe[k] = live ? (float)(ge[off] * kEps0d) : 0.f;
    if (os) os[k] = live ? (float)gs[off] : 0.f;
  }
}

// Adds the half-cell (coupling) terms of one model to the cells just outside.
__global__ void adj_ring_kernel(double* __restrict__ ge, double* __restrict__ gs, const int* __restrict__ h_cell,
                                const double* __restrict__ geps_b, const double* __restrict__ gsig_b, int ny) {
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    atomicAdd(ge + h_cell[k], geps_b[k]);
    atomicAdd(gs + h_cell[k], gsig_b[k]);
  }
}

// One block, fixed summation order: J does not depend on scheduling.
__global__ void sum_sq_kernel(const float* __restrict__ x, size_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t k = threadIdx.x; k < n; k += blockDim.x) acc += (double)x[k] * x[k];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace

// ------------------------------------------------------------------ host side

namespace {

// Device allocations of one fdtd_grad call, released together.
struct GradArena {
  std::vector<void*> ptrs;
  ~GradArena() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
      ptrs.push_back(*p);
      e = cudaMemset(*p, 0, std::max<size_t>(count, 1) * sizeof(T));
    }
    return e;
  }
};

// vjp: seed the probe terms with the device cotangent `seed` ([nsteps][nprobe])
// instead of 2 o^n (the probe energy J; J_out is then not formed);
// probe_user: device buffer for the forward pass's probe samples (null: a
// buffer of this call).
int run_grad(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
             const fdtd_probe* probes, int nprobe, int C, float* dJ_deps, float* dJ_dsig,
             float* dJ_dsrc, double* J_out, bool vjp, const float* seed, float* probe_user) {
  if (nsteps < 1 || C < 1 || nsrc < 0 || nprobe < 0 || (nsrc && !src) || (nprobe && !probes))
    return fail(ctx, FDTD_EINVAL, "fdtd_grad: bad argument");
  if (!ctx->pml_cells.empty()) return fail(ctx, FDTD_EINVAL, "fdtd_grad: not available with PML layers");
  for (int s = 0; s < nsrc; ++s)
    if (!src[s].wave) return fail(ctx, FDTD_EINVAL, "fdtd_grad: null waveform");
  if (C > nsteps) C = (int)nsteps;
  const int nsim = (int)ctx->sims.size(), ninst = (int)ctx->insts.size();
  const long long S = (nsteps + C - 1) / C;
  cudaStream_t st = ctx->stream;
  GradArena A;
  // --- forward pass with checkpoints
  float* probe_d = probe_user;
  if (!probe_d) CK(A.alloc(&probe_d, (size_t)nsteps * std::max(nprobe, 1)));
  std::vector<const float*> wv(std::max(nsrc, 1));
  for (int s = 0; s < nsrc; ++s) wv[s] = src[s].wave;
  int rc = prepare_run(ctx, nsteps, src, nsrc, wv.data(), probes, nprobe, probe_d);
  if (rc) return rc;
  std::vector<size_t> sim_off(nsim + 1, 0), inst_off(ninst + 1, 0);
  for (int s = 0; s < nsim; ++s)
    sim_off[s + 1] = sim_off[s] + (size_t)(ctx->sims[s].ny + 1) * ctx->sims[s].pitch;
  for (int k = 0; k < ninst; ++k) inst_off[k + 1] = inst_off[k] + ctx->insts[k].n;
  const size_t per_ckpt = 3 * sim_off[nsim] + inst_off[ninst];
  float* ckpt = nullptr;
  CK(A.alloc(&ckpt, per_ckpt * S));
  auto ck_field = [&](long long k, int s, int f) { return ckpt + per_ckpt * k + 3 * sim_off[s] + (size_t)f * (sim_off[s + 1] - sim_off[s]); };
  auto ck_inst = [&](long long k, int i) { return ckpt + per_ckpt * k + 3 * sim_off[nsim] + inst_off[i]; };
  for (long long k = 0; k < S; ++k) {
    const int c = ctx->cur;
    for (int s = 0; s < nsim; ++s) {
      const SimHost& sh = ctx->sims[s];
      const size_t bytes = sizeof(float) * (sim_off[s + 1] - sim_off[s]);
      CK(cudaMemcpyAsync(ck_field(k, s, 0), sh.ex[c], bytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ck_field(k, s, 1), sh.ey[c], bytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(ck_field(k, s, 2), sh.hz[c], bytes, cudaMemcpyDeviceToDevice, st));
    }
    for (int i = 0; i < ninst; ++i)
      CK(cudaMemcpyAsync(ck_inst(k, i), ctx->insts[i].state_d[c], sizeof(float) * ctx->insts[i].n,
                         cudaMemcpyDeviceToDevice, st));
    const long long base = k * C;
    CK(cudaMemcpyAsync(&ctx->run_d->base, &base, sizeof(long long), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));   // base is a host stack value
    rc = march(ctx, std::min<long long>(C, nsteps - k * C), nprobe);
    if (rc) return rc;
  }
  double* Jd = nullptr;
  CK(A.alloc(&Jd, 1));
  if (nprobe > 0 && !vjp) sum_sq_kernel<<<1, 1024, 0, st>>>(probe_d, (size_t)nsteps * nprobe, Jd);
  // --- adjoint state, frames and tables
  std::vector<AdjSimDev> asd(nsim);
  std::vector<double*> g64e(nsim), g64s(nsim);
  std::vector<float*> g32e(nsim), g32s(nsim);
  std::vector<float*> exF(nsim), eyF(nsim), hA(nsim), hB(nsim);
  for (int s = 0; s < nsim; ++s) {
    const SimHost& sh = ctx->sims[s];
    const size_t fs = sim_off[s + 1] - sim_off[s];
    AdjSimDev& a = asd[s];
    for (int p = 0; p < 2; ++p) {
      CK(A.alloc(&a.gex[p], fs));
      CK(A.alloc(&a.gey[p], fs));
      CK(A.alloc(&a.ghz[p], fs));
    }
    CK(A.alloc(&exF[s], fs * (C + 1)));
    CK(A.alloc(&eyF[s], fs * (C + 1)));
    CK(A.alloc(&hA[s], fs));
    CK(A.alloc(&hB[s], fs));
    CK(A.alloc(&g32e[s], fs));
    CK(A.alloc(&g32s[s], fs));
    CK(A.alloc(&g64e[s], fs));
    CK(A.alloc(&g64s[s], fs));
    a.exF = exF[s], a.eyF = eyF[s], a.fstride = (long long)fs;
    a.geps = g32e[s], a.gsig = g32s[s];
    a.mat = sh.mat_d;
    a.nx = sh.nx, a.ny = sh.ny, a.pitch = sh.pitch;
    a.chx = (float)(ctx->dt / (kMu0 * ctx->dy));
    a.chy = (float)(ctx->dt / (kMu0 * ctx->dx));
    a.rdy = (float)(1.0 / ctx->dy);
    a.rdx = (float)(1.0 / ctx->dx);
    a.inv_dt = (float)(1.0 / ctx->dt);
  }
  std::vector<AdjInstDev> aid(ninst);
  std::vector<float*> sF(ninst);
  std::vector<AdjWork> aw;
  size_t pre_smem = 0;
  for (int k = 0; k < ninst; ++k) {
    const Instance& in = ctx->insts[k];
    AdjInstDev& a = aid[k];
    a.M = in.map->M_d;
    CK(A.alloc(&a.gs[0], in.n));
    CK(A.alloc(&a.gs[1], in.n));
    CK(A.alloc(&sF[k], (size_t)in.map->ld * (C + 1)));   // ld: room for the two-step path's h tail
    a.sF = sF[k];
    a.y_edge = in.y_edge_d;
    a.h_cell = in.h_cell_d;
    std::vector<float> l1(in.ny), l2(in.ny);
    const double lh = 0.5 * ctx->dx * ctx->dy;   // (Dl Dl')_k on every side
    for (int e = 0; e < in.ny; ++e) {
      l1[e] = (float)(lh / ctx->dt / in.itf.dlg[e]);
      l2[e] = (float)(lh / 2 / in.itf.dlg[e]);
    }
    float* lp = nullptr;
    CK(A.alloc(&lp, 2 * (size_t)in.ny));
    CK(cudaMemcpy(lp, l1.data(), sizeof(float) * in.ny, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(lp + in.ny, l2.data(), sizeof(float) * in.ny, cudaMemcpyHostToDevice));
    a.lh_dt = lp, a.lh_2 = lp + in.ny;
    CK(A.alloc(&a.geps_b, in.ny));
    CK(A.alloc(&a.gsig_b, in.ny));
    a.n = in.n, a.ny = in.ny, a.ld = in.map->ld, a.sim = in.sim;
    for (int c0 = 0; c0 < in.n + in.ny; c0 += kPreCols)
      aw.push_back({k, c0, std::min(in.n + in.ny, c0 + kPreCols), 0});
    pre_smem = std::max(pre_smem, sizeof(float) * ((size_t)in.n + kPreCols * kPreSlices));
  }
  if (pre_smem > 48 * 1024) {
    if (pre_smem > 200 * 1024) return fail(ctx, FDTD_EINVAL, "fdtd_grad: reduced model too large");
    CK(cudaFuncSetAttribute(adj_pre_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pre_smem));
  }
  AdjSimDev* asd_d = nullptr;
  AdjInstDev* aid_d = nullptr;
  AdjWork* aw_d = nullptr;
  AdjRun* ar_d = nullptr;
  CK(A.alloc(&asd_d, nsim));
  CK(A.alloc(&aid_d, std::max(ninst, 1)));
  CK(A.alloc(&aw_d, std::max<size_t>(aw.size(), 1)));
  CK(A.alloc(&ar_d, 1));
  CK(cudaMemcpy(asd_d, asd.data(), sizeof(AdjSimDev) * nsim, cudaMemcpyHostToDevice));
  if (ninst) CK(cudaMemcpy(aid_d, aid.data(), sizeof(AdjInstDev) * ninst, cudaMemcpyHostToDevice));
  if (!aw.empty()) CK(cudaMemcpy(aw_d, aw.data(), sizeof(AdjWork) * aw.size(), cudaMemcpyHostToDevice));
  float* dsrc = dJ_dsrc;
  if (!dsrc) CK(A.alloc(&dsrc, (size_t)std::max(nsrc, 1) * nsteps));
  else CK(cudaMemsetAsync(dsrc, 0, sizeof(float) * (size_t)nsrc * nsteps, st));
  int nedges = 0;
  {
    RunDev rd;
    CK(cudaMemcpy(&rd, ctx->run_d, sizeof(RunDev), cudaMemcpyDeviceToHost));
    int2 last{0, 0};
    if (!ctx->tiles.empty())
      CK(cudaMemcpy(&last, ctx->src_range.p + ctx->tiles.size() - 1, sizeof(int2), cudaMemcpyDeviceToHost));
    nedges = last.y;
    AdjRun ar{probe_d, vjp ? seed : nullptr, ctx->probe_sim.p, ctx->probe_cell.p, ctx->src_edges.p, dsrc, nsteps, nprobe, nedges};
    CK(cudaMemcpy(ar_d, &ar, sizeof(AdjRun), cudaMemcpyHostToDevice));
  }
  // The recomputation takes two steps per launch where the context does, with
  // every model in the zone chain (FDTD_ADJ_RECOMP2=0: one step per launch):
  // the march and the zone chain also write the E frame between the two
  // sub-steps, and the chain's intermediate model state is that step's state
  // frame; 40 B per cell and pair of steps against 64.  The fields are those
  // of the one-step kernels bit for bit.
  const char* er2 = getenv("FDTD_ADJ_RECOMP2");
  MarchFn mframes = nullptr;
  if (ctx->tb && ctx->tb_march && ctx->dft_nmon == 0 && ctx->tb_tiles.size() == (size_t)ctx->tb_nchain &&
      !(er2 && atoi(er2) == 0))
    mframes = march_frames_fn(ctx->tbm_mb, ctx->tbm_ring, ctx->tbm_sparse);
  if (mframes && ctx->tbm_ring > 0)
    CK(cudaFuncSetAttribute(mframes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem(ctx->tbm_ring, 4)));
  const int npair = mframes ? C / 2 : 0;
  // per-step tables of the recomputation (frame t -> t+1), and per pair of
  // steps (frames 2p -> 2p+1 -> 2p+2), the same for every segment
  std::vector<SimDev> simtab((size_t)C * nsim), simtab2((size_t)std::max(npair, 1) * nsim);
  std::vector<RomInstDev> insttab((size_t)C * std::max(ninst, 1)),
      insttab2((size_t)std::max(npair, 1) * std::max(ninst, 1));
  {
    std::vector<SimDev> base(nsim);
    CK(cudaMemcpy(base.data(), ctx->sims_d, sizeof(SimDev) * nsim, cudaMemcpyDeviceToHost));
    std::vector<RomInstDev> ib(ninst);
    if (ninst) CK(cudaMemcpy(ib.data(), ctx->insts_d, sizeof(RomInstDev) * ninst, cudaMemcpyDeviceToHost));
    for (int t = 0; t < C; ++t) {
      for (int s = 0; s < nsim; ++s) {
        SimDev d = base[s];
        const size_t fs = sim_off[s + 1] - sim_off[s];
        d.ex[0] = exF[s] + fs * t, d.ex[1] = exF[s] + fs * (t + 1);
        d.ey[0] = eyF[s] + fs * t, d.ey[1] = eyF[s] + fs * (t + 1);
        d.hz[0] = (t & 1) ? hB[s] : hA[s];
        d.hz[1] = (t & 1) ? hA[s] : hB[s];
        simtab[(size_t)t * nsim + s] = d;
      }
      for (int k = 0; k < ninst; ++k) {
        RomInstDev d = ib[k];
        d.state[0] = sF[k] + (size_t)ctx->insts[k].map->ld * t;
        d.state[1] = sF[k] + (size_t)ctx->insts[k].map->ld * (t + 1);
        insttab[(size_t)t * ninst + k] = d;
      }
    }
    for (int p = 0; p < npair; ++p) {
      for (int s = 0; s < nsim; ++s) {
        SimDev d = base[s];
        const size_t fs = sim_off[s + 1] - sim_off[s];
        d.ex[0] = exF[s] + fs * (2 * p), d.exm = exF[s] + fs * (2 * p + 1), d.ex[1] = exF[s] + fs * (2 * p + 2);
        d.ey[0] = eyF[s] + fs * (2 * p), d.eym = eyF[s] + fs * (2 * p + 1), d.ey[1] = eyF[s] + fs * (2 * p + 2);
        d.hz[0] = (p & 1) ? hB[s] : hA[s];
        d.hz[1] = (p & 1) ? hA[s] : hB[s];
        simtab2[(size_t)p * nsim + s] = d;
      }
      for (int k = 0; k < ninst; ++k) {
        RomInstDev d = ib[k];
        const size_t ld = (size_t)ctx->insts[k].map->ld;
        d.state[0] = sF[k] + ld * (2 * p);
        d.state_mid = sF[k] + ld * (2 * p + 1);
        d.state[1] = sF[k] + ld * (2 * p + 2);
        insttab2[(size_t)p * ninst + k] = d;
      }
    }
  }
  SimDev* simtab2_d = nullptr;
  RomInstDev* insttab2_d = nullptr;
  SimDev* tail_d = nullptr;   // the one step after the pairs of an odd segment
  if (npair > 0) {
    CK(A.alloc(&simtab2_d, simtab2.size()));
    CK(A.alloc(&insttab2_d, insttab2.size()));
    CK(A.alloc(&tail_d, nsim));
    CK(cudaMemcpy(simtab2_d, simtab2.data(), sizeof(SimDev) * simtab2.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(insttab2_d, insttab2.data(), sizeof(RomInstDev) * insttab2.size(), cudaMemcpyHostToDevice));
  }
  SimDev* simtab_d = nullptr;
  RomInstDev* insttab_d = nullptr;
  RunDev* run2_d = nullptr;
  CK(A.alloc(&simtab_d, simtab.size()));
  CK(A.alloc(&insttab_d, insttab.size()));
  CK(A.alloc(&run2_d, 1));
  CK(cudaMemcpy(simtab_d, simtab.data(), sizeof(SimDev) * simtab.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(insttab_d, insttab.data(), sizeof(RomInstDev) * insttab.size(), cudaMemcpyHostToDevice));
  {
    RunDev rd;
    CK(cudaMemcpy(&rd, ctx->run_d, sizeof(RunDev), cudaMemcpyDeviceToHost));
    // the two-step kernels write the probes they own: the forward's values
    // again, into the forward's buffer; the one-step path launches no probe
    // blocks
    rd.nprobe = npair > 0 ? nprobe : 0;
    rd.probe_out = npair > 0 ? probe_d : nullptr;
    CK(cudaMemcpy(run2_d, &rd, sizeof(RunDev), cudaMemcpyHostToDevice));
  }
  const unsigned ntiles = (unsigned)ctx->tiles.size();
  // The fused cell pass: row loads in registers one row ahead (FDTD_ADJ_RING=0,
  // 167 registers, 3 CTAs per SM) or staged 1 / 2 rows ahead through shared
  // memory (FDTD_ADJ_RING=2 / 3; 4 / 3 CTAs per SM); the same arithmetic.
  int adj_ring = 0;
  if (const char* er = getenv("FDTD_ADJ_RING")) adj_ring = atoi(er) == 2 ? 2 : atoi(er) == 3 ? 3 : 0;
  auto cell_fn = adj_ring == 2 ? adj_cell_kernel<2, 4> : adj_ring == 3 ? adj_cell_kernel<3, 3> : adj_cell_kernel<0, 3>;
  const size_t cell_smem = (size_t)adj_ring * 4 * kAdjSlot4 * sizeof(float4);
  if (cell_smem > 0) CK(cudaFuncSetAttribute(cell_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem));
  // the reverse cell pass has its own tile plan (fewer resident CTAs per SM
  // than the forward kernel, so other tile heights fill whole waves)
  TileWork* atiles_d = nullptr;
  unsigned natiles = 0;
  {
    int dev = 0, nsm = 1, occ = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cell_fn, 128, cell_smem));
    const std::vector<TileWork> at = tile_table(ctx->sims, best_tile_rows(ctx->sims, (long long)nsm * std::max(occ, 1)));
    CK(A.alloc(&atiles_d, at.size()));
    CK(cudaMemcpy(atiles_d, at.data(), sizeof(TileWork) * at.size(), cudaMemcpyHostToDevice));
    natiles = (unsigned)at.size();
  }
  const int npre_extra = (nprobe + nedges + kPreCols * kPreSlices - 1) / (kPreCols * kPreSlices);
  // one fused cell pass per reverse step (FDTD_ADJ_FUSED=0: the two-pass form)
  const char* fe = getenv("FDTD_ADJ_FUSED");
  const bool fused = !(fe && atoi(fe) == 0);
  // Two reverse steps per launch (adj_march_kernel + adj_fix_kernel;
  // FDTD_ADJ_TB2=0: one step per launch): (W x kMarchOut) x th2 tiles (th2 of
  // 8..64 rows filling whole waves of resident CTAs), per warp the edges
  // whose g_E after the first step it exports (the models' interface edges,
  // the source edges).
  const char* et2 = getenv("FDTD_ADJ_TB2");
  const bool tb2 = fused && !(et2 && atoi(et2) == 0);
  TileWork* a2tiles_d = nullptr;
  unsigned na2 = 0;
  AdjMarchDev* am_d = nullptr;
  float* expv_d = nullptr;
  int* iexp_d = nullptr;
  int src_exp = 0;
  int aw2 = 4;                    // warps per CTA of adj_march_kernel
  size_t a2smem = 0;
  if (tb2) {
    {   // 3 or 4 warps per CTA: the fewer idle warps in the grids' last column blocks
      long long idle3 = 0, idle4 = 0;
      for (const SimHost& sh : ctx->sims) {
        const long long nwc = (sh.nx + kMarchOut - 1) / kMarchOut, nr = sh.ny;
        idle3 += ((nwc + 2) / 3 * 3 - nwc) * nr;
        idle4 += ((nwc + 3) / 4 * 4 - nwc) * nr;
      }
      aw2 = idle3 < idle4 ? 3 : 4;
    }
    a2smem = kAdj2SmemPerWarp * aw2;
    CK(cudaFuncSetAttribute(adj_march_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a2smem));
    if (pre_smem > 48 * 1024)
      CK(cudaFuncSetAttribute(adj_fix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pre_smem));
    int dev = 0, nsm = 1, occ = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adj_march_kernel, 32 * aw2, a2smem));
    const long long slots = (long long)nsm * std::max(occ, 1);
    const int cw = kMarchOut * aw2;   // columns per CTA
    auto tiles_for = [&](int th) {
      long long c = 0;
      for (const SimHost& sh : ctx->sims) c += (long long)((sh.nx + cw - 1) / cw) * ((sh.ny + th - 1) / th);
      return c;
    };
    int th2 = 8;
    long long best = -1;
    for (int h = 8; h <= 64; ++h) {
      const long long cost = ((tiles_for(h) + slots - 1) / slots) * (h + 3);
      if (best < 0 || cost < best) best = cost, th2 = h;
    }
    if (const char* er = getenv("FDTD_ADJ_TB2_ROWS")) th2 = std::min(4096, std::max(4, atoi(er)));
    std::vector<TileWork> t2;
    std::vector<int> tbase(nsim);
    for (int s = 0; s < nsim; ++s) {
      const SimHost& sh = ctx->sims[s];
      tbase[s] = (int)t2.size();
      for (int y0 = 0; y0 < sh.ny; y0 += th2)
        for (int x0 = 0; x0 < sh.nx; x0 += cw) t2.push_back({s, x0, y0, std::min(y0 + th2, sh.ny)});
    }
    na2 = (unsigned)t2.size();
    std::vector<std::vector<AdjExp>> lists((size_t)aw2 * t2.size());
    auto add = [&](int sim, int comp, int i, int j, int slot) {
      const SimHost& sh = ctx->sims[sim];
      const int ncx = (sh.nx + cw - 1) / cw;
      const int tile = tbase[sim] + (j / th2) * ncx + i / cw;
      lists[(size_t)aw2 * tile + (i % cw) / kMarchOut].push_back({j, i, comp, slot});
    };
    std::vector<int> iexp(std::max(ninst, 1), 0);
    int nexp = 0;
    for (int q = 0; q < ninst; ++q) {
      const Instance& in = ctx->insts[q];
      const int P = ctx->sims[in.sim].pitch;
      iexp[q] = nexp;
      for (int e = 0; e < in.ny; ++e) {
        const int code = in.y_edge[e], off = code & 0x3fffffff;
        add(in.sim, code >> 30, off % P, off / P, nexp + e);
      }
      nexp += in.ny;
    }
    src_exp = nexp;
    if (nedges > 0) {
      std::vector<SrcEdge> se(nedges);
      CK(cudaMemcpy(se.data(), ctx->src_edges.p, sizeof(SrcEdge) * nedges, cudaMemcpyDeviceToHost));
      for (int e = 0; e < nedges; ++e) add(se[e].sim, se[e].comp, se[e].i, se[e].j, nexp + e);
      nexp += nedges;
    }
    std::vector<int2> rng(lists.size());
    std::vector<AdjExp> flat;
    for (size_t w = 0; w < lists.size(); ++w) {
      std::stable_sort(lists[w].begin(), lists[w].end(), [](const AdjExp& a, const AdjExp& b) { return a.j < b.j; });
      rng[w] = make_int2((int)flat.size(), (int)(flat.size() + lists[w].size()));
      flat.insert(flat.end(), lists[w].begin(), lists[w].end());
    }
    int2* rng_d = nullptr;
    AdjExp* exp_d = nullptr;
    CK(A.alloc(&a2tiles_d, t2.size()));
    CK(A.alloc(&rng_d, rng.size()));
    CK(A.alloc(&exp_d, std::max<size_t>(flat.size(), 1)));
    CK(A.alloc(&expv_d, std::max(nexp, 1)));
    CK(A.alloc(&iexp_d, iexp.size()));
    CK(A.alloc(&am_d, 1));
    CK(cudaMemcpy(a2tiles_d, t2.data(), sizeof(TileWork) * t2.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(rng_d, rng.data(), sizeof(int2) * rng.size(), cudaMemcpyHostToDevice));
    if (!flat.empty()) CK(cudaMemcpy(exp_d, flat.data(), sizeof(AdjExp) * flat.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(iexp_d, iexp.data(), sizeof(int) * iexp.size(), cudaMemcpyHostToDevice));
    const AdjMarchDev amh{rng_d, exp_d, expv_d};
    CK(cudaMemcpy(am_d, &amh, sizeof(AdjMarchDev), cudaMemcpyHostToDevice));
  }
  // the reverse sweep's kernels launch in plain stream order (measured: 2.82
  // against 2.85 s per gradient at 16 x 1024^2 with programmatic dependent
  // launch; FDTD_ADJ_PDL=1 turns it on)
  const char* ep2 = getenv("FDTD_ADJ_PDL");
  const bool rpdl = ctx->pdl && ep2 && atoi(ep2) == 1;
  int par = 0, gpar = 0;   // the adjoint fields' and the model adjoints' current buffers
  for (long long k = S - 1; k >= 0; --k) {
    const int L = (int)std::min<long long>(C, nsteps - k * C);
    for (int s = 0; s < nsim; ++s) {
      const size_t bytes = sizeof(float) * (sim_off[s + 1] - sim_off[s]);
      CK(cudaMemcpyAsync(exF[s], ck_field(k, s, 0), bytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(eyF[s], ck_field(k, s, 1), bytes, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(hA[s], ck_field(k, s, 2), bytes, cudaMemcpyDeviceToDevice, st));
    }
    for (int i = 0; i < ninst; ++i)
      CK(cudaMemcpyAsync(sF[i], ck_inst(k, i), sizeof(float) * ctx->insts[i].n, cudaMemcpyDeviceToDevice, st));
    const long long base = k * C;
    CK(cudaMemcpyAsync(&run2_d->base, &base, sizeof(long long), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    // (programmatic dependent launch where the context uses it, as the
    // forward pass does: each kernel's launch overlaps the previous one's tail)
    int t0 = 0;
    if (npair > 0) {
      const int np = L / 2;
      for (int p = 0; p < np; ++p)
        launch_tb(ctx, st, 0, p, TbTables{simtab2_d + (size_t)p * nsim, insttab2_d + (size_t)p * ninst, run2_d, mframes});
      t0 = 2 * np;
      if (t0 < L && np > 0) {   // Hz of the last pair's output as the one-step tail's input
        std::vector<SimDev> tail(simtab.begin() + (size_t)t0 * nsim, simtab.begin() + (size_t)(t0 + 1) * nsim);
        for (int s = 0; s < nsim; ++s) {
          tail[s].hz[0] = ((np - 1) & 1) ? hA[s] : hB[s];
          tail[s].hz[1] = ((np - 1) & 1) ? hB[s] : hA[s];
        }
        CK(cudaMemcpyAsync(tail_d, tail.data(), sizeof(SimDev) * nsim, cudaMemcpyHostToDevice, st));
      }
    }
    for (int t = t0; t < L; ++t) {
      const SimDev* sdt = t > 0 && npair > 0 ? tail_d : simtab_d + (size_t)t * nsim;
      if (ctx->vec == 2)
        launch_k(yee_step_kernel<2>, ntiles, kCtaCols / 2, 0, st, ctx->pdl, sdt, (const TileWork*)ctx->tiles_d,
                 (const RunDev*)run2_d, 0, t);
      else
        launch_k(yee_step_kernel<4>, ntiles, kCtaCols / 4, 0, st, ctx->pdl, sdt, (const TileWork*)ctx->tiles_d,
                 (const RunDev*)run2_d, 0, t);
      if (ctx->nromwork + ctx->ngwork > 0)
        launch_k(rom_post_kernel, (unsigned)(ctx->nromwork + ctx->ngwork), kRomRowsPerCta * 32, ctx->post_smem, st,
                 ctx->pdl, sdt, (const RomInstDev*)(insttab_d + (size_t)t * ninst), (const RomWork*)ctx->romwork_d,
                 ctx->nromwork, (const RunDev*)run2_d, 0, t, (const GemmGroupDev*)ctx->groups_d,
                 (const GemmWork*)ctx->gwork_d, ctx->ngwork, (const int*)ctx->ginst_d);
    }
    for (int t = L - 1; t >= 0; --t) {
      const long long n = k * C + t;
      const int nb = (int)aw.size() + npre_extra;
      if (nb > 0)
        launch_k(adj_pre_kernel, (unsigned)nb, kPreCols * kPreSlices, pre_smem, st, rpdl, (const AdjSimDev*)asd_d,
                 (const AdjInstDev*)aid_d, (const AdjWork*)aw_d, (int)aw.size(), (const AdjRun*)ar_d, par, gpar, t, n);
      if (tb2 && t >= 1) {   // reverse steps t and t - 1, then the additions before t - 1
        launch_k(adj_march_kernel, na2, 32 * aw2, a2smem, st, rpdl, (const AdjSimDev*)asd_d,
                 (const TileWork*)a2tiles_d, (const AdjMarchDev*)am_d, par, t);
        if (nb > 0)
          launch_k(adj_fix_kernel, (unsigned)nb, kPreCols * kPreSlices, pre_smem, st, rpdl,
                   (const AdjSimDev*)asd_d, (const AdjInstDev*)aid_d, (const AdjWork*)aw_d, (int)aw.size(),
                   (const AdjRun*)ar_d, (const float*)expv_d, (const int*)iexp_d, src_exp, 1 - par, 1 - gpar, t - 1,
                   n - 1);
        par ^= 1;
        --t;
        continue;
      }
      gpar ^= 1;
      if (fused) {
        launch_k(cell_fn, natiles, 128, cell_smem, st, rpdl, (const AdjSimDev*)asd_d, (const TileWork*)atiles_d,
                 par, t);
      } else {
        adj_h_kernel<<<ntiles, 256, 0, st>>>(asd_d, ctx->tiles_d, par, t);
        adj_e_kernel<<<ntiles, 256, 0, st>>>(asd_d, ctx->tiles_d, par);
      }
      par ^= 1;
    }
    CK(cudaGetLastError());
    for (int s = 0; s < nsim; ++s) {
      const size_t fs = sim_off[s + 1] - sim_off[s];
      adj_flush_kernel<<<256, 256, 0, st>>>(g32e[s], g64e[s], fs);
      adj_flush_kernel<<<256, 256, 0, st>>>(g32s[s], g64s[s], fs);
    }
  }
  // half-cell terms of the coupling, then dense outputs
  for (int k = 0; k < ninst; ++k) {
    const Instance& in = ctx->insts[k];
    adj_ring_kernel<<<1, 128, 0, st>>>(g64e[in.sim], g64s[in.sim], in.h_cell_d, aid[k].geps_b,
                                        aid[k].gsig_b, in.ny);
  }
  size_t out_off = 0;
  for (int s = 0; s < nsim; ++s) {
    const SimHost& sh = ctx->sims[s];
    adj_out_kernel<<<256, 256, 0, st>>>(g64e[s], g64s[s], sh.nx, sh.ny, sh.pitch, sh.mat_d,
                                        dJ_deps ? dJ_deps + out_off : nullptr,
                                        dJ_dsig ? dJ_dsig + out_off : nullptr);
    out_off += (size_t)sh.nx * sh.ny;
  }
  CK(cudaGetLastError());
  double J = 0.0;
  CK(cudaMemcpyAsync(&J, Jd, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (J_out) *J_out = J;
  return FDTD_OK;
}

}  // namespace
