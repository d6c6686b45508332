// GB300 (sm_103a) Yee + embedded-ROM time marching: kernels, context and C ABI.
//
// Method: Zhang, Bekmambetova, Triverio, arXiv:1609.07114.  The coarse mesh
// is stepped with the integral-form Yee updates (Sec. II-A, Eqs. (3), (5));
// each embedded reduced model is stepped with its precomputed explicit map
// (Sec. IV-C, Eq. (23)).  See kernels.cuh for the data layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.hpp"
#include "kernels.cuh"

using namespace fdtdrom;

namespace {
__device__ constexpr double kMu0d = 1.25663706212e-6;   // CODATA 2018
__device__ constexpr double kEps0d = 8.8541878128e-12;
}

// ============================================================== device code

namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float comp(const float4& v, int t) {
  return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

// Programmatic dependent launch: a kernel lets the next one in the stream
// start early (pdl_trigger), and the next one runs only its prologue, which
// reads nothing the earlier kernel writes, before pdl_wait returns (the
// earlier kernel complete and its writes visible).  Both are no-ops for a
// kernel launched without the programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// E-edge coefficients from the two adjacent cells, each stored as
// {p, q} = {eps0 eps_r / dt + sigma / 2, sigma} (edge material = mean of the
// two cells, Sec. II-A): with A = eps / dt and S = sigma / 2 of the edge,
//   cb = 1 / (A + S) = 2 / (p1 + p2),   ca = (A - S) / (A + S) = 1 - (q1 + q2) / (p1 + p2),
// so r = 1 / (p1 + p2) gives both: cb = 2 r, ca = 1 - (q1 + q2) r.  On a
// lossless edge ca is exactly 1 and cb the reciprocal of A (the factor 2 and
// the halving are exact).  The reciprocal is the hardware one (one MUFU op,
// relative error ~1e-7: the same as a relative change of the edge's material
// below FP32 resolution, and the same value in every kernel).
__device__ __forceinline__ float rcp_hw(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ca and r = cb / 2; the stencils multiply r by 2/dy or 2/dx (the same bits
// as cb times 1/dy or 1/dx).
__device__ __forceinline__ void edge_coef_r(float2 m1, float2 m2, float& ca, float& r) {
  r = rcp_hw(__fadd_rn(m1.x, m2.x));
  ca = __fmaf_rn(-__fadd_rn(m1.y, m2.y), r, 1.f);
}

__device__ __forceinline__ void edge_coef(float2 m1, float2 m2, float& ca, float& cb) {
  float r;
  edge_coef_r(m1, m2, ca, r);
  cb = __fmul_rn(2.f, r);
}

// Fused coarse H and E half steps over one tile (module header).
// Each warp marches up a strip of 32 V columns x (y1 - y0) rows, keeping the
// previous row's fields and new Hz in registers; lane l owns columns
// c0 + V l .. c0 + V l + V - 1.  The first iteration recomputes the halo row
// y0 - 1 of Hz^{n+1/2}; lane 0 also recomputes the halo column c0 - 1.
// The loads of row j+1 are issued before row j is computed (two rows in
// flight per warp).
template <int V>
struct Vec;
template <>
struct Vec<4> {
  using T = float4;
  __device__ static float get(const float4& v, int t) { return comp(v, t); }
};
template <>
struct Vec<2> {
  using T = float2;
  __device__ static float get(const float2& v, int t) { return t == 0 ? v.x : v.y; }
};

template <int V>
struct RowIn {
  typename Vec<V>::T exn, eyv, hzv;  // Ex(j+1), Ey(j), Hz(j) of the lane's V columns
  float4 m4[V / 2];                  // mat(j) of the lane's V cells (2 cells per float4)
  float eyR;                         // lane 31: Ey(c0 + 32V, j)
  float exLn, eyL, hzL;              // lane 0: halo column c0 - 1
  float2 mL;
};

// dense = the row's strip holds cells other than the background bg (its
// materials are read; otherwise every cell of the strip row is bg).
template <int V>
__device__ __forceinline__ void load_row(RowIn<V>& r, const float* __restrict__ ex,
                                         const float* __restrict__ ey, const float* __restrict__ hz,
                                         const float2* __restrict__ mat, size_t row, int P, int cl,
                                         int c0, int nx, int lane, bool halo, bool dense, float2 bg) {
  using T = typename Vec<V>::T;
  r.exn = *reinterpret_cast<const T*>(ex + row + P + cl);
  r.eyv = *reinterpret_cast<const T*>(ey + row + cl);
  r.hzv = *reinterpret_cast<const T*>(hz + row + cl);
  if (dense) {
#pragma unroll
    for (int h = 0; h < V / 2; ++h) r.m4[h] = ld4(reinterpret_cast<const float*>(mat + row + cl + 2 * h));
  } else {
#pragma unroll
    for (int h = 0; h < V / 2; ++h) r.m4[h] = make_float4(bg.x, bg.y, bg.x, bg.y);
  }
  r.eyR = (lane == 31 && c0 + 32 * V <= nx) ? ey[row + c0 + 32 * V] : 0.f;
  if (halo) {
    r.exLn = ex[row + P + c0 - 1];
    r.eyL = ey[row + c0 - 1];
    r.hzL = hz[row + c0 - 1];
    r.mL = dense ? mat[row + c0 - 1] : bg;
  } else {
    r.exLn = r.eyL = r.hzL = 0.f;
    r.mL = make_float2(-1.f, 0.f);
  }
}

// Values carried from row j-1 to row j by one lane.
template <int V>
struct RowCarry {
  float exc[V];   // Ex(j) (read as the previous row's Ex(j+1))
  float hzp[V];   // Hz^{n+1/2}(j-1)
  float2 mp[V];   // mat(j-1)
  float exLc;     // lane 0: Ex(c0 - 1, j)
};

// Constants of the sparse-material path: edge coefficients between two
// background cells (the same operations as edge_coef on any other pair).
struct BgCoef {
  float ca, cy, cx;   // ca, cb / dy, cb / dx
};

// One row of the fused step for one lane (module header): Eq. (5) for Hz of
// row j, then Eq. (3) for Ex and Ey of row j, stored if j >= j0.  Every
// product and sum is an explicit correctly rounded operation, so the two
// load paths that share this function give identical bits.
template <int V>
__device__ __forceinline__ void stencil_row(const SimDev& sd, const RowIn<V>& cur, RowCarry<V>& cy,
                                            int j, int j0, int cl, int nx, int lane, bool halo,
                                            bool dcur, bool dprev, const BgCoef& bc, size_t row,
                                            float* __restrict__ hzo, float* __restrict__ exo,
                                            float* __restrict__ eyo) {
  using VT = Vec<V>;
  const unsigned FULL = 0xffffffffu;
  float2 m[V];
#pragma unroll
  for (int h = 0; h < V / 2; ++h) {
    m[2 * h] = make_float2(cur.m4[h].x, cur.m4[h].y);
    m[2 * h + 1] = make_float2(cur.m4[h].z, cur.m4[h].w);
  }
  float eyA[V + 1];
#pragma unroll
  for (int t = 0; t < V; ++t) eyA[t] = VT::get(cur.eyv, t);
  eyA[V] = __shfl_down_sync(FULL, eyA[0], 1);
  if (lane == 31) eyA[V] = cur.eyR;
  // Eq. (5): Hz^{n+1/2} = Hz^{n-1/2} + dt/(mu0 dy)(Ex_{j+1} - Ex_j)
  //                                  - dt/(mu0 dx)(Ey_{i+1} - Ey_i)
  float hn[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const bool live = (cl + t < nx) && (m[t].x >= 0.f);
    hn[t] = live ? __fsub_rn(__fmaf_rn(sd.chx, __fsub_rn(VT::get(cur.exn, t), cy.exc[t]), VT::get(cur.hzv, t)),
                             __fmul_rn(sd.chy, __fsub_rn(eyA[t + 1], eyA[t])))
                 : 0.f;
  }
  // Left neighbour of column cl: lane - 1's last cell, or the halo column.
  float hnL = __shfl_up_sync(FULL, hn[V - 1], 1);
  float2 mL;
  mL.x = __shfl_up_sync(FULL, m[V - 1].x, 1);
  mL.y = __shfl_up_sync(FULL, m[V - 1].y, 1);
  if (lane == 0) {
    mL = cur.mL;
    hnL = (halo && mL.x >= 0.f)
              ? __fsub_rn(__fmaf_rn(sd.chx, __fsub_rn(cur.exLn, cy.exLc), cur.hzL),
                          __fmul_rn(sd.chy, __fsub_rn(eyA[0], cur.eyL)))
              : 0.f;
  }
  if (j >= j0) {
    float exw[V], eyw[V];
    // Eq. (3): Ex^{n+1} = ca Ex^n + cb (Hz_j - Hz_{j-1}) / dy on edge (i, j),
    // between cells (i, j-1) and (i, j).  Rows j-1 and j both background:
    // the coefficients are the constants (warp-uniform branch).
    if (dcur || dprev) {
#pragma unroll
      for (int t = 0; t < V; ++t) {
        float v = cy.exc[t];
        if (j >= 1 && cl + t < nx && cy.mp[t].x >= 0.f && m[t].x >= 0.f) {
          float ca, r;
          edge_coef_r(cy.mp[t], m[t], ca, r);
          v = __fmaf_rn(ca, v, __fmul_rn(__fmul_rn(r, sd.rdy2), __fsub_rn(hn[t], cy.hzp[t])));
        }
        exw[t] = v;
      }
    } else {
#pragma unroll
      for (int t = 0; t < V; ++t) {
        float v = cy.exc[t];
        if (j >= 1 && cl + t < nx) v = __fmaf_rn(bc.ca, v, __fmul_rn(bc.cy, __fsub_rn(hn[t], cy.hzp[t])));
        exw[t] = v;
      }
    }
    // Ey^{n+1} = ca Ey^n - cb (Hz_i - Hz_{i-1}) / dx on edge (i, j),
    // between cells (i-1, j) and (i, j) (cell c0 - 1 is covered by the
    // strip's bit).
    if (dcur) {
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int i = cl + t;
        const float2 ml = t == 0 ? mL : m[t - 1];
        const float hl = t == 0 ? hnL : hn[t - 1];
        float v = eyA[t];
        if (i >= 1 && i < nx && ml.x >= 0.f && m[t].x >= 0.f) {
          float ca, r;
          edge_coef_r(ml, m[t], ca, r);
          v = __fmaf_rn(ca, v, -__fmul_rn(__fmul_rn(r, sd.rdx2), __fsub_rn(hn[t], hl)));
        }
        eyw[t] = v;
      }
    } else {
#pragma unroll
      for (int t = 0; t < V; ++t) {
        const int i = cl + t;
        const float hl = t == 0 ? hnL : hn[t - 1];
        float v = eyA[t];
        if (i >= 1 && i < nx) v = __fmaf_rn(bc.ca, v, -__fmul_rn(bc.cx, __fsub_rn(hn[t], hl)));
        eyw[t] = v;
      }
    }
    if constexpr (V == 4) {
      st4(hzo + row + cl, make_float4(hn[0], hn[1], hn[2], hn[3]));
      st4(exo + row + cl, make_float4(exw[0], exw[1], exw[2], exw[3]));
      st4(eyo + row + cl, make_float4(eyw[0], eyw[1], eyw[2], eyw[3]));
    } else {
      *reinterpret_cast<float2*>(hzo + row + cl) = make_float2(hn[0], hn[1]);
      *reinterpret_cast<float2*>(exo + row + cl) = make_float2(exw[0], exw[1]);
      *reinterpret_cast<float2*>(eyo + row + cl) = make_float2(eyw[0], eyw[1]);
    }
  }
#pragma unroll
  for (int t = 0; t < V; ++t) {
    cy.exc[t] = VT::get(cur.exn, t);
    cy.hzp[t] = hn[t];
    cy.mp[t] = m[t];
  }
  cy.exLc = cur.exLn;
}

// Start-of-strip state shared by both stencil kernels: the carried values
// of row js = max(j0 - 1, 0), the strip's sparse-material bit words (lane w
// holds word js/32 + w; tile heights are capped so that 32 words cover a
// tile) and the background coefficients.
template <int V>
__device__ __forceinline__ void stencil_start(const SimDev& sd, const float* __restrict__ ex, int js,
                                              int cl, int c0, int lane, bool halo, RowCarry<V>& cy,
                                              uint32_t& fw, BgCoef& bc) {
  const int P = sd.pitch;
#pragma unroll
  for (int t = 0; t < V; ++t) {
    cy.exc[t] = ex[(size_t)js * P + cl + t];
    cy.hzp[t] = 0.f;
    cy.mp[t] = make_float2(0.f, 0.f);
  }
  cy.exLc = halo ? ex[(size_t)js * P + c0 - 1] : 0.f;
  const int jb = js >> 5;
  fw = 0xffffffffu;
  if (jb + lane <= ((sd.ny - 1) >> 5)) fw = sd.mbits[(size_t)(jb + lane) * sd.nstrip + (c0 >> 7)];
  float ca, cb;
  edge_coef(sd.mbg, sd.mbg, ca, cb);
  bc.ca = ca;
  bc.cy = __fmul_rn(cb, sd.rdy);
  bc.cx = __fmul_rn(cb, sd.rdx);
}

// Whether row jj of the strip holds any non-background cell (warp-collective).
__device__ __forceinline__ bool strip_dense(uint32_t fw, int js, int jj) {
  return ((__shfl_sync(0xffffffffu, fw, (jj >> 5) - (js >> 5)) >> (jj & 31)) & 1u) != 0u;
}

// Source currents on the CTA's edges, after its rows are written:
// E^{n+1} -= cb J(t^{n+1/2}) (block-wide; every thread of the CTA calls it).
__device__ __forceinline__ void stencil_sources(const RunDev* __restrict__ run, int c,
                                                const float2* __restrict__ mat, int P,
                                                float* __restrict__ exo, float* __restrict__ eyo) {
  const int2 rg = run->src_range[blockIdx.x];
  if (rg.y > rg.x) {
    __syncthreads();
    const long long n = run->base + c;
    for (int e = rg.x + threadIdx.x; e < rg.y; e += blockDim.x) {
      const SrcEdge se = run->src_edges[e];
      const size_t off = (size_t)se.j * P + se.i;
      const float2 m2 = mat[off];
      const float2 m1 = se.comp == 0 ? mat[off - P] : mat[off - 1];
      float ca, cb;
      edge_coef(m1, m2, ca, cb);
      float* dst = se.comp == 0 ? exo : eyo;
      dst[off] = __fsub_rn(dst[off], __fmul_rn(cb, run->waves[se.src][n]));
    }
  }
}

template <int V>
__global__ void __launch_bounds__(kCtaCols / V, V == 4 ? 4 : 3)
yee_step_kernel(const SimDev* __restrict__ sims, const TileWork* __restrict__ work,
                const RunDev* __restrict__ run, int par, int c) {
  constexpr int kStrip = 32 * V;
  const TileWork tw = work[blockIdx.x];
  const SimDev sd = sims[tw.sim];
  pdl_trigger();
  pdl_wait();   // fields, run data: written by the previous kernels
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = tw.x0 + warp * kStrip;
  const int nx = sd.nx, P = sd.pitch;
  // (ternaries, not sd.ex[par]: a dynamic index would put sd in local memory)
  const float* __restrict__ ex = par ? sd.ex[1] : sd.ex[0];
  const float* __restrict__ ey = par ? sd.ey[1] : sd.ey[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  float* __restrict__ exo = par ? sd.ex[0] : sd.ex[1];
  float* __restrict__ eyo = par ? sd.ey[0] : sd.ey[1];
  float* __restrict__ hzo = par ? sd.hz[0] : sd.hz[1];
  const float2* __restrict__ mat = sd.mat;
  if (c0 < nx) {
    const int cl = c0 + V * lane;
    const int j0 = tw.y0, j1 = tw.y1;
    const int js = j0 > 0 ? j0 - 1 : 0;
    const bool halo = (lane == 0) && (c0 > 0);
    RowCarry<V> cy;
    uint32_t fw;
    BgCoef bc;
    stencil_start<V>(sd, ex, js, cl, c0, lane, halo, cy, fw, bc);
    bool dcur = strip_dense(fw, js, js), dprev = true;   // row j's bit, row j-1's bit
    RowIn<V> cur, nxt;
    load_row<V>(cur, ex, ey, hz, mat, (size_t)js * P, P, cl, c0, nx, lane, halo, dcur, sd.mbg);
    const int pf1 = run->pf1;
    for (int j = js; j < j1; ++j) {
      const size_t row = (size_t)j * P;
      const bool dn = strip_dense(fw, js, j + 1 < j1 ? j + 1 : j);
      if (pf1 > 0 && j + 1 + pf1 < j1) {   // L1 prefetch of the lane's part of a later row
        const size_t rp = row + (size_t)(1 + pf1) * P + cl;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(ex + rp + P));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(ey + rp));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(hz + rp));
        if (strip_dense(fw, js, j + 1 + pf1)) {
          asm volatile("prefetch.global.L1 [%0];" ::"l"(mat + rp));
          if (V == 4) asm volatile("prefetch.global.L1 [%0];" ::"l"(mat + rp + 2));
        }
      }
      if (j + 1 < j1) load_row<V>(nxt, ex, ey, hz, mat, row + P, P, cl, c0, nx, lane, halo, dn, sd.mbg);
      stencil_row<V>(sd, cur, cy, j, j0, cl, nx, lane, halo, dcur, dprev, bc, row, hzo, exo, eyo);
      cur = nxt;
      dprev = dcur;
      dcur = dn;
    }
  }
  stencil_sources(run, c, mat, P, exo, eyo);
}

#include "stencil_tma.cuh"

// Eq. (23) for every embedded model, then the probes.  A CTA takes
// kRomRowsPerCta rows of one model, one row per warp: v = [y; x~; h] is staged
// in shared memory and each warp forms one dot product with [P | Q] using
// float4 loads (all of a row's loads are in flight together): lane l sums
// the float4 chunks k4 = l, l + 32, ... with fused multiply-adds (x, y, z, w
// in turn), and the 32 partial sums are added by a warp xor-butterfly
// (offsets 16, 8, 4, 2, 1).
// Batched form: the simulations sharing one coupled map step it as one
// GEMM [S'] = [P | Q] [S; H], one column per simulation.  A CTA takes
// 8 RPW rows (RPW per warp) and up to 32 columns; the input panel of its
// columns is staged in shared memory column by column (ld floats each, by
// cp.async with every copy in flight at once).  Each output is formed by the
// operations of the one-row-per-warp form in the same order: lane l keeps,
// for each of the 32 columns, the partial sum of the chunks k4 = l, l + 32, ...
// of its row, and a reduce-scatter over the lanes (the butterfly's pairings,
// offsets 16, 8, 4, 2, 1) leaves column l's sum in lane l.  So both forms,
// and the two-step path's model tiles, give the same bits.  RPW = 1 gives
// more, smaller CTAs (a map shared by a few tens of simulations); RPW = 2
// reads each panel chunk for two rows (large batches).
__host__ __device__ constexpr size_t gemm_smem_floats(int ld) { return (size_t)ld * 32; }

// Asynchronous global -> shared copies (no register round trip, so every
// copy of a staging loop is in flight at once).
__device__ __forceinline__ void async_copy16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void async_copy4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// v[0..31]: this lane's partial sums of 32 columns.  Returns the total of
// column `lane` over the 32 lanes, added pairwise in the order of an xor
// butterfly with offsets 16, 8, 4, 2, 1 (floating-point addition is
// commutative, so which lane holds a pair does not change the bits).
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
  const unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; ++j) {
      const float lo = v[j], hi = v[j + o];
      const float got = __shfl_xor_sync(FULL, up ? lo : hi, o);
      v[j] = __fadd_rn(up ? hi : lo, got);
    }
  }
  return v[0];
}

// RPW rows (row pointers Mr, ld floats each, 16-B aligned) against the 32
// columns of the shared-memory panel (column c at panel + c ld); result of
// row i for column `lane` in res[i].
template <int RPW>
__device__ __forceinline__ void gemm_exact_rows(const float4* const (&Mr)[RPW], int l4, const float* panel, int ld,
                                                int lane, float (&res)[RPW]) {
  float p[RPW][32];
#pragma unroll
  for (int i = 0; i < RPW; ++i)
#pragma unroll
    for (int c = 0; c < 32; ++c) p[i][c] = 0.f;
  float4 mc[RPW];
#pragma unroll
  for (int i = 0; i < RPW; ++i) mc[i] = lane < l4 ? Mr[i][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k4 = lane; k4 < l4; k4 += 32) {
    float4 mn[RPW];
#pragma unroll
    for (int i = 0; i < RPW; ++i) mn[i] = k4 + 32 < l4 ? Mr[i][k4 + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const float4 x = *reinterpret_cast<const float4*>(panel + (size_t)c * ld + 4 * k4);
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        p[i][c] = fmaf(mc[i].x, x.x, p[i][c]);
        p[i][c] = fmaf(mc[i].y, x.y, p[i][c]);
        p[i][c] = fmaf(mc[i].z, x.z, p[i][c]);
        p[i][c] = fmaf(mc[i].w, x.w, p[i][c]);
      }
    }
#pragma unroll
    for (int i = 0; i < RPW; ++i) mc[i] = mn[i];
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) res[i] = reduce_scatter32(p[i], lane);
}

template <int RPW>
__device__ __forceinline__ void rom_gemm_rows(const SimDev* __restrict__ sims,
                                              const RomInstDev* __restrict__ insts,
                                              const GemmGroupDev g, const GemmWork gw,
                                              const int* __restrict__ ginst, int par, float* smem) {
  __shared__ const float* s_in[32];
  __shared__ float* s_out[32];
  __shared__ const float* s_hz[32];
  __shared__ const int* s_hc[32];
  __shared__ const int* s_ye[32];
  __shared__ float* s_ex[32];
  __shared__ float* s_ey[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int nwarp = kRomRowsPerCta;
  const int nc = min(32, g.B - gw.c0);
  const int ld = g.ld;
  if (tid < nc) {
    const RomInstDev ri = insts[ginst[g.inst_off + gw.c0 + tid]];
    const SimDev* sd = sims + ri.sim;
    s_in[tid] = par ? ri.state[1] : ri.state[0];
    s_out[tid] = par ? ri.state[0] : ri.state[1];
    s_hz[tid] = par ? sd->hz[0] : sd->hz[1];
    s_ex[tid] = par ? sd->ex[0] : sd->ex[1];
    s_ey[tid] = par ? sd->ey[0] : sd->ey[1];
    s_hc[tid] = ri.h_cell;
    s_ye[tid] = ri.y_edge;
  }
  const int rb = gw.r0 + RPW * warp;
  const float4* Mr[RPW];
#pragma unroll
  for (int i = 0; i < RPW; ++i)   // rows past the end repeat the last row; not stored
    Mr[i] = reinterpret_cast<const float4*>(g.M + (size_t)min(rb + i, g.n - 1) * ld);
  pdl_wait();        // model states and Hz^{n+1/2}: written by the previous kernels
  __syncthreads();   // column pointers
  float* panel = smem;   // [col][k], ld floats per column
  for (int col = warp; col < 32; col += nwarp) {
    float* pc = panel + (size_t)col * ld;
    if (col < nc) {
      const float* __restrict__ sp = s_in[col];
      const float* __restrict__ hp = s_hz[col];
      const int* __restrict__ hc = s_hc[col];
      for (int k = lane; k < g.n; k += 32) async_copy4(pc + k, sp + k);
      for (int k = g.n + lane; k < g.n + g.ny; k += 32) async_copy4(pc + k, hp + hc[k - g.n]);
      for (int k = g.n + g.ny + lane; k < ld; k += 32) pc[k] = 0.f;
    } else {
      for (int k = lane; k < ld; k += 32) pc[k] = 0.f;
    }
  }
  async_wait_all();
  __syncthreads();
  if (rb >= g.n) return;
  float res[RPW];
  gemm_exact_rows<RPW>(Mr, ld >> 2, panel, ld, lane, res);
  if (lane >= nc) return;
  float* __restrict__ so = s_out[lane];
  const int* __restrict__ ye = s_ye[lane];
  float* __restrict__ bx = s_ex[lane];
  float* __restrict__ by = s_ey[lane];
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = rb + i;
    if (r < g.n) {
      so[r] = res[i];
      if (r < g.ny) {
        const int code = ye[r];
        ((code >> 30) ? by : bx)[code & 0x3fffffff] = res[i];
      }
    }
  }
}

__global__ void __launch_bounds__(kRomRowsPerCta * 32)
rom_post_kernel(const SimDev* __restrict__ sims, const RomInstDev* __restrict__ insts,
                const RomWork* __restrict__ work, int nwork, const RunDev* __restrict__ run,
                int par, int c, const GemmGroupDev* __restrict__ groups,
                const GemmWork* __restrict__ gwork, int ngwork, const int* __restrict__ ginst) {
  extern __shared__ float4 smem4[];
  const unsigned FULL = 0xffffffffu;
  pdl_trigger();
  if ((int)blockIdx.x >= nwork && (int)blockIdx.x < nwork + ngwork) {
    const GemmWork gw = gwork[blockIdx.x - nwork];
    const GemmGroupDev g = groups[gw.group];
    if (g.rpw == 2)
      rom_gemm_rows<2>(sims, insts, g, gw, ginst, par, reinterpret_cast<float*>(smem4));
    else
      rom_gemm_rows<1>(sims, insts, g, gw, ginst, par, reinterpret_cast<float*>(smem4));
    return;
  }
  if ((int)blockIdx.x < nwork) {
    const RomWork w = work[blockIdx.x];
    const RomInstDev ri = insts[w.inst];
    const SimDev sd = sims[ri.sim];
    const float* __restrict__ s = par ? ri.state[1] : ri.state[0];
    float* __restrict__ so = par ? ri.state[0] : ri.state[1];
    const float* __restrict__ hzn = par ? sd.hz[0] : sd.hz[1];
    float* __restrict__ exo = par ? sd.ex[0] : sd.ex[1];
    float* __restrict__ eyo = par ? sd.ey[0] : sd.ey[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = w.row0 + warp;
    const bool has = r < w.row1;
    const float4* __restrict__ Mr = reinterpret_cast<const float4*>(ri.M + (size_t)(has ? r : w.row0) * ri.ld);
    const int l4 = ri.ld >> 2;
    // The first 128 float4 of this warp's row go to registers before the
    // input vector is staged, so both sets of loads are in flight together.
    constexpr int kPre = 4;
    float4 mpre[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int k = lane + 32 * u;
      mpre[u] = (has && k < l4) ? Mr[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    pdl_wait();   // model states and Hz^{n+1/2}: written by the previous kernels
    float* v = reinterpret_cast<float*>(smem4);
    for (int k = threadIdx.x; k < ri.ld; k += blockDim.x) {
      float x = 0.f;
      if (k < ri.n) x = s[k];
      else if (k < ri.n + ri.ny) x = hzn[ri.h_cell[k - ri.n]];
      v[k] = x;
    }
    __syncthreads();
    if (has) {
      float acc = 0.f;
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        const int k = lane + 32 * u;
        if (k < l4) {
          const float4 x = smem4[k];
          acc = fmaf(mpre[u].x, x.x, acc);
          acc = fmaf(mpre[u].y, x.y, acc);
          acc = fmaf(mpre[u].z, x.z, acc);
          acc = fmaf(mpre[u].w, x.w, acc);
        }
      }
      for (int k = lane + 32 * kPre; k < l4; k += 32) {
        const float4 m = Mr[k];
        const float4 x = smem4[k];
        acc = fmaf(m.x, x.x, acc);
        acc = fmaf(m.y, x.y, acc);
        acc = fmaf(m.z, x.z, acc);
        acc = fmaf(m.w, x.w, acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
      if (lane == 0) {
        so[r] = acc;
        if (r < ri.ny) {
          const int code = ri.y_edge[r];
          float* base = (code >> 30) ? eyo : exo;
          base[code & 0x3fffffff] = acc;
        }
      }
    }
  } else {
    // Probe blocks, then running-DFT blocks (one thread per monitor and
    // frequency; each accumulator has one owner, steps are stream-ordered).
    pdl_wait();
    const int b = blockIdx.x - nwork - ngwork;
    const int pb = (run->nprobe + blockDim.x - 1) / blockDim.x;
    const long long n = run->base + c;
    if (b < pb) {
      const int p = b * blockDim.x + threadIdx.x;
      if (p < run->nprobe) {
        const SimDev* sd = sims + run->probe_sim[p];
        const float* hzn = par ? sd->hz[0] : sd->hz[1];
        run->probe_out[n * run->nprobe + p] = hzn[run->probe_cell[p]];
      }
    } else {
      const int q = (b - pb) * blockDim.x + threadIdx.x;
      if (q < run->ndft) {
        const int m = q / run->nfreq, f = q - m * run->nfreq;
        const SimDev* sd = sims + run->dft_sim[m];
        const float* hzn = par ? sd->hz[0] : sd->hz[1];
        const double v = hzn[run->dft_cell[m]];
        // phase in cycles at t^{n+1/2}, reduced to [0, 1) before sin/cos
        double x = run->dft_fdt[f] * ((double)(run->step0 + n) + 0.5);
        x -= floor(x);
        double sn, cs;
        sincospi(2.0 * x, &sn, &cs);
        double2 a = run->dft_acc[q];
        a.x += v * cs;
        a.y -= v * sn;
        run->dft_acc[q] = a;
      }
    }
  }
}

// Fine-region fields from a model state, x_hat = blkdiag(V1, V2) x~ (Sec. III):
// one warp per output row, x~ staged in shared memory.  Rows [0, nE) are the
// E unknowns (all Ex then all Ey), rows [nE, nE + nH) the Hz unknowns.
__global__ void __launch_bounds__(256)
fine_fields_kernel(const float* __restrict__ V1, const float* __restrict__ V2,
                   const float* __restrict__ xt, int nE, int nH, int qE, int qH, int nEx,
                   float* __restrict__ Ex, float* __restrict__ Ey, float* __restrict__ Hz) {
  extern __shared__ float xs[];
  for (int k = threadIdx.x; k < qE + qH; k += blockDim.x) xs[k] = xt[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nE + nH; row += nw) {
    const bool e = row < nE;
    const float* __restrict__ v = e ? V1 + (size_t)row * qE : V2 + (size_t)(row - nE) * qH;
    const float* x = e ? xs : xs + qE;
    const int q = e ? qE : qH;
    float acc = 0.f;
    for (int k = lane; k < q; k += 32) acc = fmaf(v[k], x[k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      if (row < nEx) Ex[row] = acc;
      else if (e) Ey[row - nEx] = acc;
      else Hz[row - nE] = acc;
    }
  }
}

// ---- convolutional PML (open boundaries) ----------------------------------
// Run after the stencil kernel has written every cell and edge: the layer
// cells' Hz^{n+1/2} is recomputed with stretched differences, then every E
// edge next to a layer cell (its E^{n+1} used the old Hz there).  Each list
// entry is {simulation, j * pitch + i}; auxiliaries psi are per entry.
//   Hz' = Hz + dt/mu0 [ (1/ky) dEx/dy + psi_hy - (1/kx) dEy/dx - psi_hx ],
//   psi_hx = bx psi_hx + ax dEy/dx,  psi_hy = by psi_hy + ay dEx/dy.
__global__ void __launch_bounds__(256)
pml_h_kernel(const SimDev* __restrict__ sims, const PmlSimDev* __restrict__ pml,
             const int2* __restrict__ cells, int n, float* __restrict__ psi_hx,
             float* __restrict__ psi_hy, int par) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int2 ce = cells[k];
    const SimDev& sd = sims[ce.x];
    const PmlSimDev& pm = pml[ce.x];
    const int P = sd.pitch, off = ce.y, j = off / P, i = off - j * P;
    const float* ex = par ? sd.ex[1] : sd.ex[0];
    const float* ey = par ? sd.ey[1] : sd.ey[0];
    const float* hz = par ? sd.hz[1] : sd.hz[0];
    float* hzo = par ? sd.hz[0] : sd.hz[1];
    const float dEx = __fmul_rn(__fsub_rn(ex[off + P], ex[off]), sd.rdy);
    const float dEy = __fmul_rn(__fsub_rn(ey[off + 1], ey[off]), sd.rdx);
    const float py = __fmaf_rn(pm.yh[pm.nyh + j], dEx, __fmul_rn(pm.yh[j], psi_hy[k]));
    const float px = __fmaf_rn(pm.xh[pm.nxh + i], dEy, __fmul_rn(pm.xh[i], psi_hx[k]));
    psi_hy[k] = py;
    psi_hx[k] = px;
    const float d = __fsub_rn(__fadd_rn(__fmul_rn(dEx, pm.yh[2 * pm.nyh + j]), py),
                              __fadd_rn(__fmul_rn(dEy, pm.xh[2 * pm.nxh + i]), px));
    hzo[off] = __fmaf_rn(pm.dtmu, d, hz[off]);
  }
}

//   Ex' = ca Ex + cb [ (1/ky) dHz/dy + psi_ex ],  psi_ex = by psi_ex + ay dHz/dy,
//   Ey' = ca Ey - cb [ (1/kx) dHz/dx + psi_ey ],  psi_ey = bx psi_ey + ax dHz/dx.
// Entries [0, nex) are Ex edges, [nex, nex + ney) Ey edges.
__global__ void __launch_bounds__(256)
pml_e_kernel(const SimDev* __restrict__ sims, const PmlSimDev* __restrict__ pml,
             const int2* __restrict__ edges, int nex, int ney, float* __restrict__ psi_e, int par) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nex + ney; k += gridDim.x * blockDim.x) {
    const int2 ed = edges[k];
    const SimDev& sd = sims[ed.x];
    const PmlSimDev& pm = pml[ed.x];
    const int P = sd.pitch, off = ed.y, j = off / P, i = off - j * P;
    const float* hzo = par ? sd.hz[0] : sd.hz[1];
    float ca, cb;
    if (k < nex) {
      const float* ex = par ? sd.ex[1] : sd.ex[0];
      float* exo = par ? sd.ex[0] : sd.ex[1];
      const float dH = __fmul_rn(__fsub_rn(hzo[off], hzo[off - P]), sd.rdy);
      const float ps = __fmaf_rn(pm.ye[pm.nye + j], dH, __fmul_rn(pm.ye[j], psi_e[k]));
      psi_e[k] = ps;
      edge_coef(sd.mat[off - P], sd.mat[off], ca, cb);
      exo[off] = __fmaf_rn(ca, ex[off], __fmul_rn(cb, __fadd_rn(__fmul_rn(dH, pm.ye[2 * pm.nye + j]), ps)));
    } else {
      const float* ey = par ? sd.ey[1] : sd.ey[0];
      float* eyo = par ? sd.ey[0] : sd.ey[1];
      const float dH = __fmul_rn(__fsub_rn(hzo[off], hzo[off - 1]), sd.rdx);
      const float ps = __fmaf_rn(pm.xe[pm.nxe + i], dH, __fmul_rn(pm.xe[i], psi_e[k]));
      psi_e[k] = ps;
      edge_coef(sd.mat[off - 1], sd.mat[off], ca, cb);
      eyo[off] = __fmaf_rn(ca, ey[off], -__fmul_rn(cb, __fadd_rn(__fmul_rn(dH, pm.xe[2 * pm.nxe + i]), ps)));
    }
  }
}

// ---- storage function (Sec. V, Appendix A), FP64 accumulation -------------

__device__ __forceinline__ double block_sum(double v, double* red) {
  const unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = 0.0;
  if (warp == 0) {
    v = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  }
  return v;  // valid in thread 0
}

// eps0 eps_r / dt of a cell from its stored {eps0 eps_r / dt + sigma / 2, sigma}.
__device__ __forceinline__ double cell_a(float2 m) { return (double)m.x - 0.5 * (double)m.y; }

// Coarse part over one stencil tile: 1/2 eps A E^2 - dt/2 E (K H) on every
// updated edge, 1/2 mu0 A H^2 on every coarse cell.
__global__ void __launch_bounds__(256)
energy_cells_kernel(const SimDev* __restrict__ sims, const TileWork* __restrict__ work, int par,
                    double dt, double dx, double dy, double* __restrict__ partial) {
  __shared__ double red[32];
  const TileWork tw = work[blockIdx.x];
  const SimDev sd = sims[tw.sim];
  const float* __restrict__ ex = par ? sd.ex[1] : sd.ex[0];
  const float* __restrict__ ey = par ? sd.ey[1] : sd.ey[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  const float2* __restrict__ mat = sd.mat;
  const int P = sd.pitch;
  const int nxs = min(kCtaCols, sd.nx - tw.x0), nys = tw.y1 - tw.y0;
  const double area = dx * dy;
  double acc = 0.0;
  for (int k = threadIdx.x; k < nxs * nys; k += blockDim.x) {
    const int i = tw.x0 + k % nxs, j = tw.y0 + k / nxs;
    const size_t off = (size_t)j * P + i;
    const float2 m = mat[off];
    if (m.x < 0.f) continue;
    const double h = hz[off];
    acc += 0.5 * area * kMu0d * h * h;
    if (j >= 1) {
      const float2 mb = mat[off - P];
      if (mb.x >= 0.f) {
        const double e = ex[off];
        const double eps = 0.5 * (cell_a(m) + cell_a(mb)) * dt;
        acc += 0.5 * area * eps * e * e - 0.5 * dt * e * dx * (h - (double)hz[off - P]);
      }
    }
    if (i >= 1) {
      const float2 ml = mat[off - 1];
      if (ml.x >= 0.f) {
        const double e = ey[off];
        const double eps = 0.5 * (cell_a(m) + cell_a(ml)) * dt;
        acc += 0.5 * area * eps * e * e + 0.5 * dt * e * dy * (h - (double)hz[off - 1]);
      }
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// One model: dt/2 x~^T R~ x~ plus its interface half cells.
__global__ void __launch_bounds__(256)
energy_rom_kernel(const SimDev* __restrict__ sims, const RomInstDev* __restrict__ insts,
                  const EnergyInstDev* __restrict__ einst, int par, double dt,
                  double* __restrict__ partial) {
  __shared__ double red[32];
  const RomInstDev ri = insts[blockIdx.x];
  const EnergyInstDev ei = einst[blockIdx.x];
  const SimDev sd = sims[ri.sim];
  const float* __restrict__ st = par ? ri.state[1] : ri.state[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  const float* __restrict__ x = st + ri.ny;
  double acc = 0.0;
  for (int r = threadIdx.x; r < ei.q; r += blockDim.x) {
    double s = 0.0;
    const double* Rr = ei.R + (size_t)r * ei.q;
    for (int k = 0; k < ei.q; ++k) s += Rr[k] * (double)x[k];
    acc += 0.5 * dt * (double)x[r] * s;
  }
  for (int k = threadIdx.x; k < ri.ny; k += blockDim.x) {
    const double y = st[k];
    const double h = hz[ri.h_cell[k]];
    acc += ei.c1[k] * y * y - ei.c2[k] * y * h;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Per simulation: sum of its tiles' and models' partial sums.
__global__ void __launch_bounds__(256)
energy_sum_kernel(const double* __restrict__ tile_part, const int* __restrict__ tile_base,
                  const double* __restrict__ inst_part, const RomInstDev* __restrict__ insts,
                  int ninst, double* __restrict__ out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int t = tile_base[s] + threadIdx.x; t < tile_base[s + 1]; t += blockDim.x) acc += tile_part[t];
  for (int k = threadIdx.x; k < ninst; k += blockDim.x)
    if (insts[k].sim == s) acc += inst_part[k];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[s] = acc;
}

__global__ void advance_kernel(RunDev* run, int by) {
  if (threadIdx.x == 0 && blockIdx.x == 0) run->base += by;
}

}  // namespace

#include "tb.cuh"
#include "tb_march.cuh"

// ============================================================== host side

namespace fdtdrom {

static std::mutex g_err_mu;
static std::string g_err;

int set_global_error(int code, const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = msg;
  return code;
}

}  // namespace fdtdrom

namespace {

constexpr int kChunk = 16;  // steps per captured graph (even: parity repeats)
constexpr int kNoOverride = -1000;   // a tuner override not set

struct SimHost {
  int nx = 0, ny = 0, pitch = 0;
  std::vector<double> eps_r, sigma;
  std::vector<unsigned char> region;   // 1 = cell covered by a reduced model
  std::vector<float2> mat;
  float* ex[2] = {nullptr, nullptr};
  float* ey[2] = {nullptr, nullptr};
  float* hz[2] = {nullptr, nullptr};
  float2* mat_d = nullptr;
  float2 mbg = {0.f, 0.f};                // background material (sparse-material bits)
  int nstrip = 0;                         // 128-column strips per row
  std::vector<uint32_t> mbits;
  uint32_t* mbits_d = nullptr;
  bool all_dense = false;
  int tile_base = 0, ncx = 0, ncy = 0, th = 0;   // tiles: ncx x ncy of kCtaCols x th cells
};

// Background of a simulation: the most frequent material among up to 4096
// cells sampled on a regular stride (none when no value repeats, i.e. every
// strip row is read densely).
bool pick_background(const SimHost& sh, float2* bg) {
  std::map<uint64_t, int> cnt;
  const long long ncell = (long long)sh.nx * sh.ny;
  const long long stride = std::max<long long>(1, ncell / 4096);
  for (long long k = 0; k < ncell; k += stride) {
    const float2 m = sh.mat[(size_t)(k / sh.nx) * sh.pitch + (k % sh.nx)];
    uint64_t key;
    std::memcpy(&key, &m, sizeof(key));
    ++cnt[key];
  }
  uint64_t best = 0;
  int bc = 0;
  for (const auto& kv : cnt)
    if (kv.second > bc) best = kv.first, bc = kv.second;
  if (bc < 2) return false;
  std::memcpy(bg, &best, sizeof(best));
  return true;
}

// Recompute the sparse-material bits of rows [ja, jb).
void update_mbits(SimHost& sh, int ja, int jb) {
  const uint64_t* m = reinterpret_cast<const uint64_t*>(sh.mat.data());
  uint64_t bgk;
  std::memcpy(&bgk, &sh.mbg, sizeof(bgk));
  for (int j = ja; j < jb; ++j)
    for (int st = 0; st < sh.nstrip; ++st) {
      bool dense = sh.all_dense;
      const int i0 = std::max(st * 128 - 1, 0), i1 = std::min(st * 128 + 128, sh.nx);
      for (int i = i0; i < i1 && !dense; ++i) dense = m[(size_t)j * sh.pitch + i] != bgk;
      uint32_t& w = sh.mbits[(size_t)(j >> 5) * sh.nstrip + st];
      const uint32_t bit = 1u << (j & 31);
      w = dense ? (w | bit) : (w & ~bit);
    }
}

// The run-time map of one (model, interface materials) pair.  Instances of
// the same model whose outside half cells carry identical materials share it
// (one copy of [P | Q] in HBM/L2 for a whole batch).
struct CoupledMap {
  long long model_id = 0;
  std::vector<double> key;   // dplus, dminus, dlg of the interface
  la::Mat P, Q;
  int ld = 0;
  float* M_d = nullptr;      // [P | Q | 0] FP32, n x ld
  double* R_d = nullptr;     // R~ (q x q, FP64) for the storage function
  double* c_d = nullptr;     // c1 (ny) then c2 (ny)
  ~CoupledMap() {
    cudaFree(M_d);
    cudaFree(R_d);
    cudaFree(c_d);
  }
};

struct Instance {
  int sim = 0, i0 = 0, j0 = 0, a = 0, b = 0, q = 0, ny = 0, n = 0;
  InterfaceDesc itf;
  std::shared_ptr<CoupledMap> map;
  float* state_d[3] = {nullptr, nullptr, nullptr};   // ping-pong pair, mid-step vector (ld floats each)
  int* y_edge_d = nullptr;
  int* h_cell_d = nullptr;
  std::vector<int> y_edge, h_cell;
};

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t reserve(size_t n) {
    if (n <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) cap = std::max<size_t>(n, 1);
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct fdtd_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  double dx = 0, dy = 0, dt = 0;
  std::vector<SimHost> sims;
  std::vector<TileWork> tiles;
  int vec = 4;                     // columns per lane of the stencil kernel (2 or 4)
  bool stencil_tma = false;        // bulk-copy (TMA) ring form of the stencil (V = 4)
  bool pdl = true;                 // programmatic dependent launch of the step kernels (FDTD_PDL=0: off)
  int pf1 = 0;                     // one-step stencil: rows prefetched into L1 ahead (FDTD_PF1)
  unsigned* status_d = nullptr;    // kernels' status word (RunDev::status)
  SimDev* sims_d = nullptr;
  TileWork* tiles_d = nullptr;
  std::vector<Instance> insts;
  RomInstDev* insts_d = nullptr;
  RomWork* romwork_d = nullptr;
  int nromwork = 0;
  GemmGroupDev* groups_d = nullptr;   // batched form of shared maps
  GemmWork* gwork_d = nullptr;
  int* ginst_d = nullptr;
  int ngwork = 0;
  size_t post_smem = 0;
  RunDev* run_d = nullptr;
  EnergyInstDev* einst_d = nullptr;
  DevBuf<double> energy_scratch;   // per-tile and per-model partial sums, per-sim totals
  int* tile_base_d = nullptr;      // nsim + 1 tile offsets
  DevBuf<int2> src_range;
  DevBuf<SrcEdge> src_edges;
  DevBuf<const float*> waves;
  DevBuf<int> probe_sim, probe_cell;
  DevBuf<float> host_waves, host_probes;
  // sources and probes the device lists were last built for (prepare_run;
  // empty: rebuild), and the pinned slots the run record and wave pointers
  // are copied from (a copy from pinned memory does not wait for the stream)
  std::vector<long long> run_sig;
  // sources (waveforms left out) and probes of the most recent fdtd_run /
  // fdtd_run_host: the autotuner times its candidates with them
  std::vector<fdtd_source> last_src;
  std::vector<fdtd_probe> last_prb;
  struct RunSlot {
    unsigned char* host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;   // recorded after the slot's copies
  };
  RunSlot run_slots[4];
  int run_slot_next = 0;
  // convolutional PML (fdtd_set_pml): per simulation its descriptor and
  // coefficient arrays, and the concatenated cell / edge lists of all
  // simulations with their auxiliaries
  std::vector<fdtd_pml_desc> pml_desc;          // ncells = 0: none
  std::vector<std::vector<float>> pml_coef;     // per sim: xh | yh | xe | ye
  std::vector<int2> pml_cells, pml_edges;       // edges: all Ex entries, then all Ey
  int pml_nex = 0;
  DevBuf<float> pml_coef_d;
  DevBuf<PmlSimDev> pml_sims_d;
  DevBuf<int2> pml_cells_d, pml_edges_d;
  DevBuf<float> pml_psi;                        // hx | hy (per cell), e (per edge)
  // device FP32 copies of model bases (fdtd_fine_fields), per model id
  struct Basis {
    long long id;
    float* V1;
    float* V2;
  };
  std::vector<Basis> bases;
  // running DFT monitors (fdtd_dft_set)
  int dft_nmon = 0, dft_nfreq = 0;
  DevBuf<int> dft_sim, dft_cell;
  DevBuf<double> dft_fdt;
  DevBuf<double2> dft_acc;
  int cur = 0;
  long long step = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_nprobe_blocks[2] = {-1, -1};
  // two-steps-per-launch path (tb.cuh)
  bool tb = false;
  std::vector<TbTile> tb_tiles;       // ordinary tiles then one per model
  std::vector<int> tb_base;           // per simulation: first ordinary tile
  std::vector<int4> tb_zones;
  TbTile* tb_tiles_d = nullptr;
  size_t tb_tiles_cap = 0;
  int4* tb_zones_d = nullptr;
  TbRun* tb_run_d = nullptr;
  DevBuf<SrcEdge> tb_src;
  DevBuf<int> tb_prb;
  cudaGraphExec_t tb_graph[2] = {nullptr, nullptr};
  int tb_graph_nprobe[2] = {-1, -1};
  // zone chain (tb.cuh zone_step_kernel / rom_chain_kernel): the last
  // tb_nchain model tiles step their maps outside the tile, on a side stream
  // of the highest priority forked from the context's stream per pair
  int tb_chain_mode = 1;           // FDTD_TB_CHAIN at creation: 0 never, 1 every model, 2 (-1) shared maps
  std::vector<char> in_gemm;       // per instance: stepped in a GEMM group (upload_instances)
  int tb_nchain = 0;
  int chain_nrow = 0;              // rom_chain_kernel blocks stepping single models (romwork prefix)
  size_t zone_smem = 0, chain_smem = 0;
  DevBuf<float> zone_scratch;
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int prio_hi = 0;
  // row-marching form of the two-step path (tb_march.cuh): ordinary areas in
  // yee_tb2m_kernel, tb_tiles then holds only the model tiles
  int tb_mode = -1;                // FDTD_TB at creation: 0 off, 1 on where it applies, -1 automatic
  bool tb_march = false;
  std::vector<TileWork> tbm_tiles;
  std::vector<int2> tbm_zone_rng;
  std::vector<int4> tbm_zones;
  TileWork* tbm_tiles_d = nullptr;
  int2* tbm_zone_rng_d = nullptr;
  int4* tbm_zones_d = nullptr;
  TbMarchDev* tbm_d = nullptr;
  DevBuf<int2> tbm_src_rng, tbm_prb_rng;
  DevBuf<int> tbm_ent_sim;
  DevBuf<MarchSrc> tbm_src;
  DevBuf<MarchPrb> tbm_prb;
  int tbm_th = 0;
  int tbm_pf = 0;                  // rows prefetched ahead of the loads (FDTD_TB_PF: > 0 into L2, < 0 into L1)
  int tbm_mb = 4;                  // resident CTAs per SM the kernel is compiled for (FDTD_TB_MB)
  int tbm_ring = 0;                // rows staged ahead through shared memory (FDTD_TB_RING; 0: registers)
  int tbm_w = 4;                   // warps per CTA, 3 or 4 (kMarchOut columns each)
  bool tbm_sparse = false;         // some simulation has a background material (sparse-material form)
  // configuration chosen by fdtd_autotune (0: the fixed rule or the
  // environment): one-step tile rows, row-marching tile rows, simulations per
  // shared map from which it steps as a GEMM, GEMM rows per warp
  int ov_th1 = 0, ov_thm = 0, ov_gemm_min = 0, ov_rpw = 0, ov_ring = -1, ov_pf = kNoOverride, ov_mb = 0;
  // measurement mode (fdtd_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double t_yee = 0, t_post = 0;
  long long n_yee = 0, n_post = 0;
  std::string err;
};

namespace {

int fail(fdtd_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  set_global_error(code, msg);
  return code;
}

#define CK(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(ctx, FDTD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// After a synchronisation: FDTD_ETIMEOUT (and the word cleared) if a
// kernel's bounded wait gave up since the last check.
int check_status(fdtd_ctx* ctx) {
  unsigned st = 0;
  CK(cudaMemcpy(&st, ctx->status_d, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st) {
    CK(cudaMemset(ctx->status_d, 0, sizeof(unsigned)));
    return fail(ctx, FDTD_ETIMEOUT, "a kernel's bounded wait for its staged rows gave up; results are invalid");
  }
  return FDTD_OK;
}

// NVTX range for the duration of a scope (profiler timelines).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

void drop_graphs(fdtd_ctx* ctx) {
  for (int p = 0; p < 2; ++p) {
    if (ctx->graph[p]) cudaGraphExecDestroy(ctx->graph[p]);
    ctx->graph[p] = nullptr;
    ctx->graph_nprobe_blocks[p] = -1;
    if (ctx->tb_graph[p]) cudaGraphExecDestroy(ctx->tb_graph[p]);
    ctx->tb_graph[p] = nullptr;
    ctx->tb_graph_nprobe[p] = -1;
  }
}

// Plan of the two-steps-per-pass path: one tile per model whose output is
// the model's zone (yee_tb2_kernel), and for the rest either the row-marching
// kernel's (W x kMarchOut) x th tiles (default) or, with FDTD_TB_SMEM=1, ordinary
// kTbW x kTbH shared-memory tiles of yee_tb2_kernel (issue-bound: measured
// 118 against 186 Gcell-steps/s for the one-step kernel at 4096^2); and the
// zone lists.  The path is used only when every model fits the in-CTA model
// step and no model lies within reach (two steps plus the zone margin) of
// another's tile.
int plan_tb(fdtd_ctx* ctx) {
  ctx->run_sig.clear();   // the per-run lists follow the plan
  ctx->tb = false;
  ctx->tb_march = false;
  ctx->tb_nchain = 0;
  ctx->tb_tiles.clear();
  ctx->tb_zones.clear();
  ctx->tbm_tiles.clear();
  ctx->tbm_zone_rng.clear();
  ctx->tbm_zones.clear();
  // FDTD_TB=0: off; 1: on wherever it applies; unset: the row-marching form
  // where it applies, unless a fused model tile (one CTA stepping a model
  // twice between the sub-steps) would make the pair of steps slower than two
  // one-step launches.  Estimates, measured on GB300: the march 5.8 ps per
  // cell and pair, a fused model tile 0.6 ns per element of [P | Q] plus
  // 5 us, a one-step launch at least 3.5 us (5.3 ps per cell) plus 4.5 us for
  // the model launch.  With every model in the zone chain (the default) two
  // steps per launch measured faster at every size tried: 128^2 with a q = 400
  // model 6.9 against 8.1 us per step, 1024^2 with a q = 400 model 7.9
  // against 10.9, 1536^2 with 8 q = 200 models 11.1 against 11.4, the
  // 4096^2 benchmark grid 342.8 against 188.2 Gcell-steps/s.  The march
  // reads the materials of background-only strip rows as the one-step
  // kernel does, so grids of sparse scatterers take it too.  fdtd_autotune
  // times both choices.
  const int mode = ctx->tb_mode;
  if (mode == 0) return FDTD_OK;
  if (!ctx->pml_cells.empty()) return FDTD_OK;   // the layers' corrections need the one-step form
  const char* es = getenv("FDTD_TB_SMEM");
  const bool march = !(mode == 1 && es && atoi(es) == 1);
  // Models whose map is stepped outside their zone tile (zone chain):
  // FDTD_TB_CHAIN=1 (default) every model, 0 none, 2 those whose map is
  // shared by a GEMM group (one [P | Q] panel applied to many simulations'
  // vectors).  Measured on GB300 (Gcell-steps/s, best tile height of each):
  // every model chained 342.8 / 384.0 / 321.1 / 290.5 on the 4096^2 grid,
  // the 8192^2 lattice, 256 batched grids and 16 x 1024^2, against 314.8 /
  // 384.2 / 321.3 / 258.7 with only the shared maps and 315.1 / 349.3 /
  // 272.0 / 258.5 with none: the chain spreads a model over many CTAs,
  // where a fused tile holds one CTA for the whole map.
  const size_t ninst = ctx->insts.size();
  std::vector<char> chain(ninst, 0);
  for (size_t k = 0; k < ninst; ++k)
    chain[k] = ctx->tb_chain_mode == 1 ||
               (ctx->tb_chain_mode < 0 && k < ctx->in_gemm.size() && ctx->in_gemm[k]);
  if (mode != 1) {
    double cells = 0, fused_us = 0;
    for (const SimHost& sh : ctx->sims) cells += (double)sh.nx * sh.ny;
    for (size_t k = 0; k < ninst; ++k)
      if (!chain[k]) fused_us = std::max(fused_us, 0.6e-3 * ctx->insts[k].n * (double)ctx->insts[k].map->ld + 5.0);
    if (fused_us > 0.0) {
      const double two = std::max(5.8e-6 * cells, fused_us);
      const double one = 2.0 * (std::max(5.3e-6 * cells, 3.5) + 4.5);
      if (two >= one) return FDTD_OK;
    }
  }
  const int M = kTbZoneMargin;
  std::vector<int4> zone(ninst);
  for (size_t k = 0; k < ninst; ++k) {
    const Instance& in = ctx->insts[k];
    const SimHost& sh = ctx->sims[in.sim];
    if (in.map->ld > kTbMaxRomN && !chain[k]) return FDTD_OK;
    // columns rounded out to multiples of 4 (whole float4 groups of the march)
    int4 z{std::max(in.i0 - M, 0) & ~3, std::max(in.j0 - M, 0), std::min((in.i0 + in.a + M + 3) & ~3, sh.nx),
           std::min(in.j0 + in.b + M, sh.ny)};
    if ((z.z - (z.x & ~3)) + 4 + 2 > kTbSW - 2 || z.w - z.y > kTbH) return FDTD_OK;
    zone[k] = z;
  }
  for (size_t k = 0; k < ctx->insts.size(); ++k)
    for (size_t m = 0; m < ctx->insts.size(); ++m) {
      if (k == m || ctx->insts[k].sim != ctx->insts[m].sim) continue;
      const Instance& o = ctx->insts[m];
      const int4 w{zone[k].x - M, zone[k].y - M, zone[k].z + M, zone[k].w + M};   // tile's reach
      if (!(o.i0 + o.a + 1 <= w.x || o.i0 - 1 >= w.z || o.j0 + o.b + 1 <= w.y || o.j0 - 1 >= w.w))
        return FDTD_OK;
    }
  ctx->tb_base.assign(ctx->sims.size(), 0);
  if (march) {
    // (W x kMarchOut) x th tiles, 8 <= th <= 64; th fills whole waves of
    // resident CTAs: minimise ceil(T / slots) * (th + 3) (three rows of
    // sub-step halo).  Fused model tiles run beside the first wave; each
    // takes the registers of two of this kernel's CTAs, so those slots are
    // left to them.  Measured on GB300: tiles taller than 64 rows (one
    // under-filled wave) lose on large grids (8192^2 lattice: 357 rows 284,
    // 64 rows 384 Gcell-steps/s), and a partial last wave costs a whole one
    // (4096^2: 64 rows, 576 tiles, 342.8; 48 rows, 774 tiles, 295.9).
    int dev = 0, nsm = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // compiled for 4 resident CTAs (128 registers, no spills; measured 300.7
    // against 280.1 Gcell-steps/s for 3 CTAs at 162 registers, 4096^2)
    ctx->tbm_mb = 4;
    if (const char* em = getenv("FDTD_TB_MB")) ctx->tbm_mb = atoi(em) == 3 ? 3 : 4;
    if (ctx->ov_mb) ctx->tbm_mb = ctx->ov_mb;
    // the sparse-material form where some strip row holds only background
    // material (a background alone, e.g. the vacuum rings of random grids,
    // saves nothing: every strip row is read)
    ctx->tbm_sparse = false;
    for (const SimHost& sh : ctx->sims) {
      if (sh.all_dense || ctx->tbm_sparse) continue;
      for (int j = 0; j < sh.ny && !ctx->tbm_sparse; ++j)
        for (int st = 0; st < sh.nstrip && !ctx->tbm_sparse; ++st)
          ctx->tbm_sparse = ((sh.mbits[(size_t)(j >> 5) * sh.nstrip + st] >> (j & 31)) & 1u) == 0u;
    }
    // loads through a ring of rows in shared memory: by default for the
    // sparse form (its register form needs more than the 128 registers of
    // 4 CTAs per SM; 8192^2 lattice: 0.342 ms per launch with a ring of 2
    // against 0.459 with registers)
    ctx->tbm_ring = ctx->tbm_sparse ? 2 : 0;
    if (const char* eg = getenv("FDTD_TB_RING")) ctx->tbm_ring = std::min(4, std::max(0, atoi(eg)));
    if (ctx->ov_ring >= 0) ctx->tbm_ring = ctx->ov_ring;
    if (ctx->tbm_ring == 1 || ctx->tbm_mb == 3) ctx->tbm_ring = 0;
    // 3 or 4 warps per CTA (kMarchOut columns each): whichever leaves fewer
    // warps idle in the grids' last column blocks (FDTD_TB_WARPS overrides);
    // 1024 columns are 9 warp columns: three CTAs of three warps
    {
      long long idle3 = 0, idle4 = 0;
      for (const SimHost& sh : ctx->sims) {
        const long long nwc = (sh.nx + kMarchOut - 1) / kMarchOut;
        idle3 += ((nwc + 2) / 3 * 3 - nwc) * sh.ny;
        idle4 += ((nwc + 3) / 4 * 4 - nwc) * sh.ny;
      }
      ctx->tbm_w = idle3 < idle4 ? 3 : 4;
      if (const char* ew = getenv("FDTD_TB_WARPS")) ctx->tbm_w = atoi(ew) == 3 ? 3 : 4;
    }
    const int cw = kMarchOut * ctx->tbm_w;   // columns per CTA
    if (ctx->tbm_ring > 0)
      CK(cudaFuncSetAttribute(march_fn(4, ctx->tbm_ring, ctx->tbm_sparse),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem(ctx->tbm_ring, 4)));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, march_fn(ctx->tbm_mb, ctx->tbm_ring, ctx->tbm_sparse),
                                                  32 * ctx->tbm_w, march_smem(ctx->tbm_ring, ctx->tbm_w));
    long long nfused = 0;
    for (size_t k = 0; k < ninst; ++k) nfused += chain[k] ? 0 : 1;
    const long long slots = std::max((long long)nsm, (long long)nsm * std::max(occ, 1) - 2 * nfused);
    auto tiles_for = [&](int th) {
      long long t = 0;
      for (const SimHost& sh : ctx->sims)
        t += (long long)((sh.nx + cw - 1) / cw) * ((sh.ny + th - 1) / th);
      return t;
    };
    int th = 8;
    long long best = -1;
    for (int h = 8; h <= 64; ++h) {
      const long long cost = ((tiles_for(h) + slots - 1) / slots) * (h + 3);
      if (best < 0 || cost < best) best = cost, th = h;
    }
    if (const char* er = getenv("FDTD_TB_ROWS")) th = std::min(4096, std::max(4, atoi(er)));
    if (ctx->ov_thm) th = ctx->ov_thm;
    // Rows prefetched ahead of the register loads: FDTD_TB_PF = d > 0 into L2
    // (a bulk prefetch), d < 0 into L1 (per lane), 0 none.  Default: L1, two
    // rows ahead (measured on GB300, 4096^2: 0.0961 ms per launch against
    // 0.1065 without, 0.1063 / 0.1014 / 0.1047 one / three / four rows ahead).
    ctx->tbm_pf = -2;
    if (const char* ep = getenv("FDTD_TB_PF")) ctx->tbm_pf = std::min(16, std::max(-8, atoi(ep)));
    if (ctx->ov_pf != kNoOverride) ctx->tbm_pf = ctx->ov_pf;
    ctx->tbm_th = th;
    for (int s = 0; s < (int)ctx->sims.size(); ++s) {
      const SimHost& sh = ctx->sims[s];
      ctx->tb_base[s] = (int)ctx->tbm_tiles.size();
      for (int y0 = 0; y0 < sh.ny; y0 += th)
        for (int x0 = 0; x0 < sh.nx; x0 += cw) {
          const TileWork t{s, x0, y0, std::min(y0 + th, sh.ny)};
          int2 zr{(int)ctx->tbm_zones.size(), 0};
          for (size_t k = 0; k < ctx->insts.size(); ++k) {
            if (ctx->insts[k].sim != s) continue;
            const int4 z = zone[k];
            if (z.x < x0 + cw && z.z > x0 && z.y < t.y1 && z.w > t.y0) ctx->tbm_zones.push_back(z);
          }
          zr.y = (int)ctx->tbm_zones.size();
          ctx->tbm_tiles.push_back(t);
          ctx->tbm_zone_rng.push_back(zr);
        }
    }
    cudaFree(ctx->tbm_tiles_d);
    cudaFree(ctx->tbm_zone_rng_d);
    cudaFree(ctx->tbm_zones_d);
    ctx->tbm_tiles_d = nullptr;
    ctx->tbm_zone_rng_d = nullptr;
    ctx->tbm_zones_d = nullptr;
    const size_t nt = ctx->tbm_tiles.size();
    CK(cudaMalloc(&ctx->tbm_tiles_d, sizeof(TileWork) * nt));
    CK(cudaMemcpy(ctx->tbm_tiles_d, ctx->tbm_tiles.data(), sizeof(TileWork) * nt, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->tbm_zone_rng_d, sizeof(int2) * nt));
    CK(cudaMemcpy(ctx->tbm_zone_rng_d, ctx->tbm_zone_rng.data(), sizeof(int2) * nt, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->tbm_zones_d, sizeof(int4) * std::max<size_t>(ctx->tbm_zones.size(), 1)));
    if (!ctx->tbm_zones.empty())
      CK(cudaMemcpy(ctx->tbm_zones_d, ctx->tbm_zones.data(), sizeof(int4) * ctx->tbm_zones.size(),
                    cudaMemcpyHostToDevice));
    if (!ctx->tbm_d) CK(cudaMalloc(&ctx->tbm_d, sizeof(TbMarchDev)));
    ctx->tb_march = true;
  } else {
    for (int s = 0; s < (int)ctx->sims.size(); ++s) {
      const SimHost& sh = ctx->sims[s];
      ctx->tb_base[s] = (int)ctx->tb_tiles.size();
      for (int y0 = 0; y0 < sh.ny; y0 += kTbH)
        for (int x0 = 0; x0 < sh.nx; x0 += kTbW) {
          TbTile t{s, x0, std::min(x0 + kTbW, sh.nx), y0, std::min(y0 + kTbH, sh.ny), -1, 0, 0, 0, 0, 0, 0};
          t.zone_b = (int)ctx->tb_zones.size();
          for (size_t k = 0; k < ctx->insts.size(); ++k) {
            if (ctx->insts[k].sim != s) continue;
            const int4 z = zone[k];
            if (z.x < t.x1 && z.z > t.x0 && z.y < t.y1 && z.w > t.y0) ctx->tb_zones.push_back(z);
          }
          t.zone_e = (int)ctx->tb_zones.size();
          ctx->tb_tiles.push_back(t);
        }
    }
  }
  // model tiles: the fused ones first, then the zone chain's (each with its
  // window's scratch: Ex, Ey, Hz after the first sub-step)
  size_t scr = 0, zsm = 0, csm = 0;
  ctx->tb_nchain = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (size_t k = 0; k < ninst; ++k) {
      if ((int)chain[k] != pass) continue;
      const int4 z = zone[k];
      TbTile t{ctx->insts[k].sim, z.x, z.z, z.y, z.w, (int)k, 0, 0, 0, 0, 0, 0, 0};
      if (pass == 1) {
        const size_t nf = (size_t)zone_rows(z.y, z.w) * 4 * zone_sw4(z.x, z.z);
        t.scr = (int)(scr / 4);
        scr += 3 * nf;
        zsm = std::max(zsm, sizeof(float) * 5 * nf);
        const int ld = ctx->insts[k].map->ld;
        csm = std::max(csm, sizeof(float) * (k < ctx->in_gemm.size() && ctx->in_gemm[k] ? gemm_smem_floats(ld)
                                                                                          : (size_t)ld));
        ++ctx->tb_nchain;
      }
      ctx->tb_tiles.push_back(t);
    }
  ctx->chain_nrow = 0;
  if (ctx->tb_nchain > 0) {
    if (scr > (size_t)INT32_MAX * 4) return fail(ctx, FDTD_EINVAL, "zone scratch too large");
    CK(ctx->zone_scratch.reserve(scr));
    // single models of the chain are the one-step path's row-per-warp work
    // (every model outside a GEMM group); shared maps its GEMM tiles
    if (ctx->tb_chain_mode == 1) ctx->chain_nrow = ctx->nromwork;
    ctx->zone_smem = zsm;
    ctx->chain_smem = csm;
    if (zsm > 200 * 1024 || csm > 200 * 1024) return fail(ctx, FDTD_EINVAL, "zone chain too large for shared memory");
    CK(cudaFuncSetAttribute(zone_step_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
    CK(cudaFuncSetAttribute(zone_step_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
    CK(cudaFuncSetAttribute(rom_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(csm, (size_t)16)));
    if (!ctx->side_stream) {
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      ctx->prio_hi = hi;
      CK(cudaStreamCreateWithPriority(&ctx->side_stream, cudaStreamNonBlocking, hi));
      CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
  }
  cudaFree(ctx->tb_zones_d);
  ctx->tb_zones_d = nullptr;
  if (!ctx->tb_zones.empty()) {
    CK(cudaMalloc(&ctx->tb_zones_d, sizeof(int4) * ctx->tb_zones.size()));
    CK(cudaMemcpy(ctx->tb_zones_d, ctx->tb_zones.data(), sizeof(int4) * ctx->tb_zones.size(), cudaMemcpyHostToDevice));
  }
  if (!ctx->tb_run_d) CK(cudaMalloc(&ctx->tb_run_d, sizeof(TbRun)));
  const size_t smem = kTbSmemFields;
  CK(cudaFuncSetAttribute(yee_tb2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ctx->tb = true;
  return FDTD_OK;
}

// Instances are stepped either one row per warp (rom_post_kernel's first
// block range) or, when at least FDTD_ROM_GEMM_MIN (default 20) of them share
// one coupled map, as one GEMM over the shared [P | Q] (second range; 8 or
// 16 rows x up to 32 simulations per CTA, FDTD_GEMM_RPW = 1 or 2).  Both
// forms give the same bits.
int upload_instances(fdtd_ctx* ctx) {
  std::vector<RomInstDev> h(ctx->insts.size());
  std::vector<RomWork> wk;
  size_t smem = 0;
  int gemm_min = 20;   // measured: below ~20 simulations per map one row per warp is as fast or faster
  if (const char* e = getenv("FDTD_ROM_GEMM_MIN")) gemm_min = std::max(1, atoi(e));
  if (ctx->ov_gemm_min) gemm_min = ctx->ov_gemm_min;
  // rows per warp of the GEMM form: 2 when the map is shared by >= 32
  // simulations (the panel is re-staged less often), else 1 (more CTAs);
  // FDTD_GEMM_RPW = 1 or 2 overrides (same results, speed only)
  int rpw_env = 0;
  if (const char* e = getenv("FDTD_GEMM_RPW")) rpw_env = atoi(e) == 2 ? 2 : 1;
  if (ctx->ov_rpw) rpw_env = ctx->ov_rpw;
  std::vector<const CoupledMap*> maps;
  std::vector<std::vector<int>> members;
  for (size_t k = 0; k < ctx->insts.size(); ++k) {
    const CoupledMap* m = ctx->insts[k].map.get();
    size_t g = 0;
    while (g < maps.size() && maps[g] != m) ++g;
    if (g == maps.size()) maps.push_back(m), members.emplace_back();
    members[g].push_back((int)k);
  }
  std::vector<GemmGroupDev> groups;
  std::vector<GemmWork> gwork;
  std::vector<int> ginst;
  std::vector<char> in_gemm(ctx->insts.size(), 0);
  for (size_t g = 0; g < maps.size(); ++g) {
    if ((int)members[g].size() < gemm_min) continue;
    const int gemm_rpw = rpw_env ? rpw_env : ((int)members[g].size() >= 32 ? 2 : 1);
    // the GEMM's shared-memory panel must fit one CTA; else row per warp
    if (sizeof(float) * gemm_smem_floats(maps[g]->ld) > 200 * 1024) continue;
    const Instance& in0 = ctx->insts[members[g][0]];
    GemmGroupDev gd{maps[g]->M_d, in0.n, in0.ny, maps[g]->ld, (int)members[g].size(), (int)ginst.size(), gemm_rpw, 0, 0};
    for (int k : members[g]) ginst.push_back(k), in_gemm[k] = 1;
    for (int r0 = 0; r0 < gd.n; r0 += gemm_rpw * kRomRowsPerCta)
      for (int c0 = 0; c0 < gd.B; c0 += 32) gwork.push_back({(int)groups.size(), r0, c0, 0});
    groups.push_back(gd);
    smem = std::max(smem, sizeof(float) * gemm_smem_floats(gd.ld));
  }
  for (size_t k = 0; k < ctx->insts.size(); ++k) {
    const Instance& in = ctx->insts[k];
    RomInstDev& d = h[k];
    d.M = in.map->M_d;
    d.state[0] = in.state_d[0], d.state[1] = in.state_d[1], d.state_mid = in.state_d[2];
    d.y_edge = in.y_edge_d, d.h_cell = in.h_cell_d;
    d.n = in.n, d.ny = in.ny, d.ld = in.map->ld, d.sim = in.sim;
    if (in_gemm[k]) continue;
    for (int r0 = 0; r0 < in.n; r0 += kRomRowsPerCta)
      wk.push_back({(int)k, r0, std::min(in.n, r0 + kRomRowsPerCta), 0});
    smem = std::max(smem, sizeof(float) * (size_t)in.map->ld);
  }
  cudaFree(ctx->groups_d);
  cudaFree(ctx->gwork_d);
  cudaFree(ctx->ginst_d);
  ctx->groups_d = nullptr;
  ctx->gwork_d = nullptr;
  ctx->ginst_d = nullptr;
  ctx->ngwork = (int)gwork.size();
  if (!groups.empty()) {
    CK(cudaMalloc(&ctx->groups_d, sizeof(GemmGroupDev) * groups.size()));
    CK(cudaMemcpy(ctx->groups_d, groups.data(), sizeof(GemmGroupDev) * groups.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->gwork_d, sizeof(GemmWork) * gwork.size()));
    CK(cudaMemcpy(ctx->gwork_d, gwork.data(), sizeof(GemmWork) * gwork.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->ginst_d, sizeof(int) * ginst.size()));
    CK(cudaMemcpy(ctx->ginst_d, ginst.data(), sizeof(int) * ginst.size(), cudaMemcpyHostToDevice));
  }
  if (ctx->insts_d) cudaFree(ctx->insts_d);
  if (ctx->romwork_d) cudaFree(ctx->romwork_d);
  if (ctx->einst_d) cudaFree(ctx->einst_d);
  ctx->insts_d = nullptr;
  ctx->romwork_d = nullptr;
  ctx->einst_d = nullptr;
  if (!h.empty()) {
    std::vector<EnergyInstDev> eh(ctx->insts.size());
    for (size_t k = 0; k < ctx->insts.size(); ++k) {
      const Instance& in = ctx->insts[k];
      eh[k] = {in.map->R_d, in.map->c_d, in.map->c_d + in.ny, in.q, in.sim, 0, 0};
    }
    CK(cudaMalloc(&ctx->einst_d, sizeof(EnergyInstDev) * eh.size()));
    CK(cudaMemcpy(ctx->einst_d, eh.data(), sizeof(EnergyInstDev) * eh.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->insts_d, sizeof(RomInstDev) * h.size()));
    CK(cudaMemcpy(ctx->insts_d, h.data(), sizeof(RomInstDev) * h.size(), cudaMemcpyHostToDevice));
    if (!wk.empty()) {
      CK(cudaMalloc(&ctx->romwork_d, sizeof(RomWork) * wk.size()));
      CK(cudaMemcpy(ctx->romwork_d, wk.data(), sizeof(RomWork) * wk.size(), cudaMemcpyHostToDevice));
    }
  }
  ctx->nromwork = (int)wk.size();
  ctx->in_gemm = in_gemm;
  ctx->post_smem = smem;
  if (smem > 48 * 1024) {
    if (smem > 200 * 1024) return fail(ctx, FDTD_EINVAL, "reduced model too large for one CTA's shared memory");
    CK(cudaFuncSetAttribute(rom_post_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  drop_graphs(ctx);
  return plan_tb(ctx);
}

// Launch with the programmatic-serialisation attribute when pdl is set (the
// kernel's prologue may overlap the previous kernel's tail; see pdl_wait).
// The priority form sets the launch's scheduling priority (kept by a graph
// node captured from it).
template <typename... KArgs, typename... Args>
void launch_k(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, bool pdl,
              int prio, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (prio != 0) {
    at[na].id = cudaLaunchAttributePriority;
    at[na].val.priority = prio;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  cudaLaunchKernelEx(&cfg, k, args...);
}
template <typename... KArgs, typename... Args>
void launch_k(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, bool pdl,
              Args... args) {
  launch_k(k, grid, block, smem, s, pdl, 0, args...);
}

void launch_yee(fdtd_ctx* ctx, cudaStream_t s, int par, int c) {
  const unsigned nb = (unsigned)ctx->tiles.size();
  if (ctx->stencil_tma)
    yee_step_tma_kernel<<<nb, kCtaCols / 4, kTmaSmem, s>>>(ctx->sims_d, ctx->tiles_d, ctx->run_d, par, c);
  else if (ctx->vec == 2)
    launch_k(yee_step_kernel<2>, nb, kCtaCols / 2, 0, s, ctx->pdl, (const SimDev*)ctx->sims_d,
             (const TileWork*)ctx->tiles_d, (const RunDev*)ctx->run_d, par, c);
  else
    launch_k(yee_step_kernel<4>, nb, kCtaCols / 4, 0, s, ctx->pdl, (const SimDev*)ctx->sims_d,
             (const TileWork*)ctx->tiles_d, (const RunDev*)ctx->run_d, par, c);
}

// PML corrections of one step (after the stencil, before the model maps).
void launch_pml(fdtd_ctx* ctx, cudaStream_t s, int par) {
  const int nc = (int)ctx->pml_cells.size(), ne = (int)ctx->pml_edges.size();
  if (nc == 0) return;
  float* psi = ctx->pml_psi.p;
  pml_h_kernel<<<std::min(1024, (nc + 255) / 256), 256, 0, s>>>(ctx->sims_d, ctx->pml_sims_d.p,
                                                                ctx->pml_cells_d.p, nc, psi, psi + nc, par);
  if (ne > 0)
    pml_e_kernel<<<std::min(1024, (ne + 255) / 256), 256, 0, s>>>(
        ctx->sims_d, ctx->pml_sims_d.p, ctx->pml_edges_d.p, ctx->pml_nex, ne - ctx->pml_nex, psi + 2 * nc, par);
}

// Launches one step (chunk index c) on stream s.
void launch_step(fdtd_ctx* ctx, cudaStream_t s, int par, int c, int nprobe_blocks) {
  launch_yee(ctx, s, par, c);
  launch_pml(ctx, s, par);
  const int nb = ctx->nromwork + ctx->ngwork + nprobe_blocks;
  if (nb > 0)
    launch_k(rom_post_kernel, (unsigned)nb, kRomRowsPerCta * 32, ctx->post_smem, s,
             ctx->pdl, (const SimDev*)ctx->sims_d,
             (const RomInstDev*)ctx->insts_d,
             (const RomWork*)ctx->romwork_d, ctx->nromwork, (const RunDev*)ctx->run_d, par, c,
             (const GemmGroupDev*)ctx->groups_d, (const GemmWork*)ctx->gwork_d, ctx->ngwork,
             (const int*)ctx->ginst_d);
}

int ensure_graph(fdtd_ctx* ctx, int par, int nprobe_blocks) {
  if (ctx->graph[par] && ctx->graph_nprobe_blocks[par] == nprobe_blocks) return FDTD_OK;
  if (ctx->graph[par]) cudaGraphExecDestroy(ctx->graph[par]);
  ctx->graph[par] = nullptr;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
  for (int c = 0; c < kChunk; ++c) launch_step(ctx, ctx->capture_stream, par ^ (c & 1), c, nprobe_blocks);
  advance_kernel<<<1, 32, 0, ctx->capture_stream>>>(ctx->run_d, kChunk);
  CK(cudaStreamEndCapture(ctx->capture_stream, &g));
  cudaError_t e = cudaGraphInstantiate(&ctx->graph[par], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, FDTD_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  ctx->graph_nprobe_blocks[par] = nprobe_blocks;
  return FDTD_OK;
}

// Whether cell (i, j) of simulation sim lies in one of its PML layers.
bool pml_cell(const fdtd_ctx* ctx, int sim, int i, int j) {
  if (sim >= (int)ctx->pml_desc.size()) return false;
  const fdtd_pml_desc& d = ctx->pml_desc[sim];
  if (d.sides == 0 || d.ncells == 0) return false;
  const SimHost& sh = ctx->sims[sim];
  const int n = d.ncells;
  return ((d.sides & FDTD_PML_W) && i < n) || ((d.sides & FDTD_PML_E) && i >= sh.nx - n) ||
         ((d.sides & FDTD_PML_S) && j < n) || ((d.sides & FDTD_PML_N) && j >= sh.ny - n);
}

// Whether an E edge is recomputed by the PML kernels (a cell beside it is a
// layer cell).
bool pml_edge(const fdtd_ctx* ctx, int sim, int comp, int i, int j) {
  if (comp == 0) return pml_cell(ctx, sim, i, j - 1) || pml_cell(ctx, sim, i, j);
  return pml_cell(ctx, sim, i - 1, j) || pml_cell(ctx, sim, i, j);
}

bool edge_updated(const SimHost& s, int comp, int i, int j) {
  if (comp == 0) {
    if (i < 0 || i >= s.nx || j < 1 || j > s.ny - 1) return false;
    return !s.region[(size_t)(j - 1) * s.nx + i] && !s.region[(size_t)j * s.nx + i];
  }
  if (j < 0 || j >= s.ny || i < 1 || i > s.nx - 1) return false;
  return !s.region[(size_t)j * s.nx + i - 1] && !s.region[(size_t)j * s.nx + i];
}

// Uploads the per-run source and probe tables (wave pointers already device).
RunDev run_record(const fdtd_ctx* ctx, long long nsteps, float* probe_out, int nprobe);

// The run record and the wave pointer table, copied in stream order from the
// next pinned slot (reused once its previous copies have completed).
int upload_run(fdtd_ctx* ctx, const RunDev& rd, const float* const* wave_dev, int nsrc) {
  fdtd_ctx::RunSlot& sl = ctx->run_slots[ctx->run_slot_next];
  ctx->run_slot_next = (ctx->run_slot_next + 1) % 4;
  if (sl.done) CK(cudaEventSynchronize(sl.done));
  else CK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  const size_t off = (sizeof(RunDev) + 15) & ~(size_t)15;
  const size_t bytes = off + sizeof(float*) * (size_t)std::max(nsrc, 1);
  if (sl.cap < bytes) {
    if (sl.host) CK(cudaFreeHost(sl.host));
    sl.host = nullptr;
    sl.cap = 0;
    CK(cudaHostAlloc((void**)&sl.host, bytes, cudaHostAllocDefault));
    sl.cap = bytes;
  }
  std::memcpy(sl.host, &rd, sizeof(RunDev));
  cudaStream_t st = ctx->stream;
  if (nsrc > 0) {
    std::memcpy(sl.host + off, wave_dev, sizeof(float*) * nsrc);
    CK(cudaMemcpyAsync(ctx->waves.p, sl.host + off, sizeof(float*) * nsrc, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(ctx->run_d, sl.host, sizeof(RunDev), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(sl.done, st));
  return FDTD_OK;
}

// Uploads the per-run source and probe tables (wave pointers already
// device).  The tables depend only on where the sources and probes sit and on
// the plan, so when a run repeats the previous run's (a problem driven chunk
// by chunk) they are kept and only the run record and the wave pointers are
// copied; neither copy waits for the stream.
int prepare_run(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
                const float* const* wave_dev, const fdtd_probe* probes, int nprobe,
                float* probe_out) {
  std::vector<long long> sig;
  sig.reserve(2 + 5 * (size_t)nsrc + 3 * (size_t)nprobe);
  sig.push_back(nsrc);
  for (int s = 0; s < nsrc; ++s) {
    const fdtd_source& so = src[s];
    sig.insert(sig.end(), {(long long)so.sim, (long long)so.comp, (long long)so.i, (long long)so.j, (long long)so.len});
  }
  sig.push_back(nprobe);
  for (int p = 0; p < nprobe; ++p) sig.insert(sig.end(), {(long long)probes[p].sim, (long long)probes[p].i, (long long)probes[p].j});
  if (nprobe > 0 && !probe_out) return fail(ctx, FDTD_EINVAL, "fdtd_run: probe_out is NULL");
  if (!ctx->run_sig.empty() && sig == ctx->run_sig) {
    for (int s = 0; s < nsrc; ++s)
      if (!wave_dev[s]) return fail(ctx, FDTD_EINVAL, "fdtd_run: malformed source " + std::to_string(s));
    return upload_run(ctx, run_record(ctx, nsteps, probe_out, nprobe), wave_dev, nsrc);
  }
  ctx->run_sig.clear();
  const int ntiles = (int)ctx->tiles.size();
  std::vector<std::vector<SrcEdge>> per(ntiles);
  std::vector<unsigned char> seen;
  for (int s = 0; s < nsrc; ++s) {
    const fdtd_source& so = src[s];
    if (so.sim < 0 || so.sim >= (int)ctx->sims.size() || (so.comp != 0 && so.comp != 1) ||
        so.len < 1 || !wave_dev[s])
      return fail(ctx, FDTD_EINVAL, "fdtd_run: malformed source " + std::to_string(s));
    const SimHost& sh = ctx->sims[so.sim];
    for (int t = 0; t < so.len; ++t) {
      const int i = so.comp == 0 ? so.i + t : so.i;
      const int j = so.comp == 0 ? so.j : so.j + t;
      if (!edge_updated(sh, so.comp, i, j))
        return fail(ctx, FDTD_EINVAL, "fdtd_run: source " + std::to_string(s) +
                                          " drives a PEC, interface or covered edge");
      if (pml_edge(ctx, so.sim, so.comp, i, j))
        return fail(ctx, FDTD_EINVAL, "fdtd_run: source " + std::to_string(s) + " drives an edge next to a PML cell");
      const int tile = sh.tile_base + (j / sh.th) * sh.ncx + i / kCtaCols;
      for (const SrcEdge& o : per[tile])
        if (o.sim == so.sim && o.comp == so.comp && o.i == i && o.j == j)
          return fail(ctx, FDTD_EINVAL, "fdtd_run: two sources drive the same edge");
      per[tile].push_back({so.sim, so.comp, i, j, s, {0, 0, 0}});
    }
  }
  std::vector<int2> range(ntiles);
  std::vector<SrcEdge> edges;
  for (int t = 0; t < ntiles; ++t) {
    range[t].x = (int)edges.size();
    edges.insert(edges.end(), per[t].begin(), per[t].end());
    range[t].y = (int)edges.size();
  }
  std::vector<int> psim(nprobe), pcell(nprobe);
  for (int p = 0; p < nprobe; ++p) {
    const fdtd_probe& pr = probes[p];
    if (pr.sim < 0 || pr.sim >= (int)ctx->sims.size())
      return fail(ctx, FDTD_EINVAL, "fdtd_run: probe sim out of range");
    const SimHost& sh = ctx->sims[pr.sim];
    if (pr.i < 0 || pr.i >= sh.nx || pr.j < 0 || pr.j >= sh.ny)
      return fail(ctx, FDTD_EINVAL, "fdtd_run: probe outside the grid");
    psim[p] = pr.sim;
    pcell[p] = pr.j * sh.pitch + pr.i;
  }
  CK(ctx->src_range.reserve(ntiles));
  CK(ctx->src_edges.reserve(edges.size()));
  CK(ctx->waves.reserve(std::max(nsrc, 1)));
  CK(ctx->probe_sim.reserve(std::max(nprobe, 1)));
  CK(ctx->probe_cell.reserve(std::max(nprobe, 1)));
  cudaStream_t st = ctx->stream;
  CK(cudaMemcpyAsync(ctx->src_range.p, range.data(), sizeof(int2) * ntiles, cudaMemcpyHostToDevice, st));
  if (!edges.empty())
    CK(cudaMemcpyAsync(ctx->src_edges.p, edges.data(), sizeof(SrcEdge) * edges.size(), cudaMemcpyHostToDevice, st));
  if (nprobe > 0) {
    CK(cudaMemcpyAsync(ctx->probe_sim.p, psim.data(), sizeof(int) * nprobe, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->probe_cell.p, pcell.data(), sizeof(int) * nprobe, cudaMemcpyHostToDevice, st));
  }
  if (ctx->tb) {   // per-tile source and probe lists of the two-step path
    const int nt = (int)ctx->tb_tiles.size();
    std::vector<std::vector<SrcEdge>> ts(nt);
    std::vector<std::vector<int>> tp(nt);
    const int first_rom_tile = nt - (int)ctx->insts.size();
    const int W = ctx->tbm_w, cw = kMarchOut * W;
    const int nw = ctx->tb_march ? W * (int)ctx->tbm_tiles.size() : 0;
    std::vector<std::vector<MarchSrc>> ms(nw);
    std::vector<std::vector<MarchPrb>> mq(nw);
    const int th = ctx->tbm_th;
    for (const SrcEdge& e : edges) {
      const SimHost& sh = ctx->sims[e.sim];
      if (ctx->tb_march) {
        // every warp whose computed columns [c0 - 4, c0 + 124) and rows
        // [max(y0 - 2, 0), min(y1, ny)] hold the edge; c0 = 120 k
        const int ncx = (sh.nx + cw - 1) / cw, ncy = (sh.ny + th - 1) / th;
        for (int ty = std::max(0, e.j / th - 1); ty <= std::min(ncy - 1, (e.j + 2) / th); ++ty) {
          const int y0 = ty * th, y1 = std::min(y0 + th, sh.ny);
          if (e.j < std::max(y0 - 2, 0) || e.j > std::min(y1, sh.ny)) continue;
          for (int k = std::max(0, (e.i + 4) / kMarchOut - 1); k <= (e.i + 4) / kMarchOut; ++k) {
            const int c0 = kMarchOut * k;
            if (c0 >= sh.nx || e.i < c0 - 4 || e.i >= c0 + 124) continue;
            const int t = ctx->tb_base[e.sim] + ty * ncx + k / W;
            ms[W * t + k % W].push_back({e.j, e.i, e.comp | (e.src << 1), 0.f});
          }
        }
      } else {
        const int ncx = (sh.nx + kTbW - 1) / kTbW, ncy = (sh.ny + kTbH - 1) / kTbH;
        for (int ty = std::max(0, (e.j - 1) / kTbH); ty <= std::min(ncy - 1, (e.j + 1) / kTbH); ++ty)
          for (int tx = std::max(0, (e.i - 1) / kTbW); tx <= std::min(ncx - 1, (e.i + 1) / kTbW); ++tx) {
            const int t = ctx->tb_base[e.sim] + ty * ncx + tx;
            const TbTile& tt = ctx->tb_tiles[t];
            if (e.i >= tt.x0 - 1 && e.i <= tt.x1 && e.j >= tt.y0 - 1 && e.j <= tt.y1) ts[t].push_back(e);
          }
      }
      for (int t = first_rom_tile; t < nt; ++t) {
        const TbTile& tt = ctx->tb_tiles[t];
        if (tt.sim == e.sim && e.i >= tt.x0 - 1 && e.i <= tt.x1 && e.j >= tt.y0 - 1 && e.j <= tt.y1)
          ts[t].push_back(e);
      }
    }
    for (int p = 0; p < nprobe; ++p) {
      const int sim = psim[p], i = probes[p].i, j = probes[p].j;
      int owner = -1;
      for (int t = first_rom_tile; t < nt; ++t) {
        const TbTile& tt = ctx->tb_tiles[t];
        if (tt.sim == sim && i >= tt.x0 && i < tt.x1 && j >= tt.y0 && j < tt.y1) owner = t;
      }
      if (owner >= 0) {
        tp[owner].push_back(p);
        continue;
      }
      const SimHost& sh = ctx->sims[sim];
      if (ctx->tb_march) {
        const int ncx = (sh.nx + cw - 1) / cw;
        const int t = ctx->tb_base[sim] + (j / th) * ncx + i / cw;
        mq[W * t + (i % cw) / kMarchOut].push_back({j, i, p, 0});
      } else {
        tp[ctx->tb_base[sim] + (j / kTbH) * ((sh.nx + kTbW - 1) / kTbW) + i / kTbW].push_back(p);
      }
    }
    std::vector<SrcEdge> fs;
    std::vector<int> fp;
    for (int t = 0; t < nt; ++t) {
      TbTile& tt = ctx->tb_tiles[t];
      tt.src_b = (int)fs.size();
      fs.insert(fs.end(), ts[t].begin(), ts[t].end());
      tt.src_e = (int)fs.size();
      tt.prb_b = (int)fp.size();
      fp.insert(fp.end(), tp[t].begin(), tp[t].end());
      tt.prb_e = (int)fp.size();
    }
    CK(ctx->tb_src.reserve(fs.size()));
    CK(ctx->tb_prb.reserve(fp.size()));
    if (nt > 0 && (!ctx->tb_tiles_d || ctx->tb_tiles_cap < ctx->tb_tiles.size())) {
      cudaFree(ctx->tb_tiles_d);
      ctx->tb_tiles_d = nullptr;
      CK(cudaMalloc(&ctx->tb_tiles_d, sizeof(TbTile) * ctx->tb_tiles.size()));
      ctx->tb_tiles_cap = ctx->tb_tiles.size();
    }
    if (nt > 0) CK(cudaMemcpyAsync(ctx->tb_tiles_d, ctx->tb_tiles.data(), sizeof(TbTile) * nt, cudaMemcpyHostToDevice, st));
    if (!fs.empty()) CK(cudaMemcpyAsync(ctx->tb_src.p, fs.data(), sizeof(SrcEdge) * fs.size(), cudaMemcpyHostToDevice, st));
    if (!fp.empty()) CK(cudaMemcpyAsync(ctx->tb_prb.p, fp.data(), sizeof(int) * fp.size(), cudaMemcpyHostToDevice, st));
    TbRun tr{ctx->tb_zones_d, ctx->tb_src.p, ctx->tb_prb.p};
    CK(cudaMemcpyAsync(ctx->tb_run_d, &tr, sizeof(TbRun), cudaMemcpyHostToDevice, st));
    if (ctx->tb_march) {   // per-warp lists, rows ascending
      std::vector<int2> srng(nw), prng(nw);
      std::vector<MarchSrc> fms;
      std::vector<MarchPrb> fmq;
      std::vector<int> fsim;
      for (int w = 0; w < nw; ++w) {
        std::stable_sort(ms[w].begin(), ms[w].end(), [](const MarchSrc& a, const MarchSrc& b) {
          return a.j != b.j ? a.j < b.j : (a.cs & 1) < (b.cs & 1);
        });
        std::stable_sort(mq[w].begin(), mq[w].end(), [](const MarchPrb& a, const MarchPrb& b) { return a.j < b.j; });
        srng[w] = make_int2((int)fms.size(), (int)(fms.size() + ms[w].size()));
        fms.insert(fms.end(), ms[w].begin(), ms[w].end());
        fsim.insert(fsim.end(), ms[w].size(), ctx->tbm_tiles[w / W].sim);
        prng[w] = make_int2((int)fmq.size(), (int)(fmq.size() + mq[w].size()));
        fmq.insert(fmq.end(), mq[w].begin(), mq[w].end());
      }
      CK(ctx->tbm_src_rng.reserve(nw));
      CK(ctx->tbm_prb_rng.reserve(nw));
      CK(ctx->tbm_src.reserve(fms.size()));
      CK(ctx->tbm_prb.reserve(fmq.size()));
      CK(cudaMemcpyAsync(ctx->tbm_src_rng.p, srng.data(), sizeof(int2) * nw, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(ctx->tbm_prb_rng.p, prng.data(), sizeof(int2) * nw, cudaMemcpyHostToDevice, st));
      CK(ctx->tbm_ent_sim.reserve(fsim.size()));
      if (!fms.empty()) {
        CK(cudaMemcpyAsync(ctx->tbm_src.p, fms.data(), sizeof(MarchSrc) * fms.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ctx->tbm_ent_sim.p, fsim.data(), sizeof(int) * fsim.size(), cudaMemcpyHostToDevice, st));
        const int ne = (int)fms.size();
        march_src_cb_kernel<<<(ne + 127) / 128, 128, 0, st>>>(ctx->sims_d, ctx->tbm_ent_sim.p, ctx->tbm_src.p, ne);
        CK(cudaGetLastError());
      }
      if (!fmq.empty())
        CK(cudaMemcpyAsync(ctx->tbm_prb.p, fmq.data(), sizeof(MarchPrb) * fmq.size(), cudaMemcpyHostToDevice, st));
      const TbMarchDev tmd{ctx->tbm_src_rng.p, ctx->tbm_src.p, ctx->tbm_prb_rng.p, ctx->tbm_prb.p,
                           ctx->tbm_zone_rng_d, ctx->tbm_zones_d};
      CK(cudaMemcpyAsync(ctx->tbm_d, &tmd, sizeof(TbMarchDev), cudaMemcpyHostToDevice, st));
    }
  }
  const int rc = upload_run(ctx, run_record(ctx, nsteps, probe_out, nprobe), wave_dev, nsrc);
  if (rc) return rc;
  ctx->run_sig = std::move(sig);
  return FDTD_OK;
}

// The run record of a run of nsteps from the current step.
RunDev run_record(const fdtd_ctx* ctx, long long nsteps, float* probe_out, int nprobe) {
  RunDev rd{};
  rd.base = 0;
  rd.nsteps = nsteps;
  rd.waves = ctx->waves.p;
  rd.src_range = ctx->src_range.p;
  rd.src_edges = ctx->src_edges.p;
  rd.probe_out = probe_out;
  rd.probe_sim = ctx->probe_sim.p;
  rd.probe_cell = ctx->probe_cell.p;
  rd.nprobe = nprobe;
  rd.ndft = ctx->dft_nmon * ctx->dft_nfreq;
  rd.step0 = ctx->step;
  rd.dft_fdt = ctx->dft_fdt.p;
  rd.dft_sim = ctx->dft_sim.p;
  rd.dft_cell = ctx->dft_cell.p;
  rd.dft_acc = ctx->dft_acc.p;
  rd.nfreq = ctx->dft_nfreq;
  rd.pf1 = ctx->pf1;
  rd.status = ctx->status_d;
  return rd;
}

void launch_tb(fdtd_ctx* ctx, cudaStream_t s, int par, int c);

// Blocks of rom_post after the model rows: probes, then DFT monitors.
int post_extra_blocks(const fdtd_ctx* ctx, int nprobe) {
  constexpr int t = kRomRowsPerCta * 32;
  return (nprobe + t - 1) / t + (ctx->dft_nmon * ctx->dft_nfreq + t - 1) / t;
}

// Sums the elapsed times of the recorded event triples (yee, post).
int drain_events(fdtd_ctx* ctx) {
  for (int k = 0; k + 2 < ctx->ev_used; k += 3) {
    CK(cudaEventSynchronize(ctx->ev[k + 2]));
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, ctx->ev[k], ctx->ev[k + 1]));
    CK(cudaEventElapsedTime(&b, ctx->ev[k + 1], ctx->ev[k + 2]));
    ctx->t_yee += a;
    ctx->t_post += b;
  }
  ctx->ev_used = 0;
  return FDTD_OK;
}

int march_timed(fdtd_ctx* ctx, long long nsteps, int nprobe) {
  const int nprobe_blocks = post_extra_blocks(ctx, nprobe);
  const bool post = ctx->nromwork + ctx->ngwork + nprobe_blocks > 0;
  while ((int)ctx->ev.size() < 3 * 64) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    ctx->ev.push_back(e);
  }
  long long t = 0;
  if (ctx->tb && ctx->dft_nmon == 0) {   // pairs of steps in one stencil launch
    for (; t + 2 <= nsteps; t += 2) {
      const int par = ctx->cur ^ (int)(t & 1);
      cudaEvent_t* e = &ctx->ev[ctx->ev_used];
      CK(cudaEventRecord(e[0], ctx->stream));
      launch_tb(ctx, ctx->stream, par, 0);
      CK(cudaEventRecord(e[1], ctx->stream));
      CK(cudaEventRecord(e[2], ctx->stream));
      advance_kernel<<<1, 32, 0, ctx->stream>>>(ctx->run_d, 2);
      CK(cudaGetLastError());
      ctx->n_yee += 1;   // one launch of two steps
      ctx->ev_used += 3;
      if (ctx->ev_used == (int)ctx->ev.size()) {
        int rc = drain_events(ctx);
        if (rc) return rc;
      }
    }
  }
  for (; t < nsteps; ++t) {
    const int par = ctx->cur ^ (int)(t & 1);
    cudaEvent_t* e = &ctx->ev[ctx->ev_used];
    CK(cudaEventRecord(e[0], ctx->stream));
    // the step index for sources/probes is base + c with base = 0 here
    launch_yee(ctx, ctx->stream, par, 0);
    launch_pml(ctx, ctx->stream, par);
    CK(cudaEventRecord(e[1], ctx->stream));
    if (post)
      rom_post_kernel<<<ctx->nromwork + ctx->ngwork + nprobe_blocks, kRomRowsPerCta * 32, ctx->post_smem,
                        ctx->stream>>>(ctx->sims_d, ctx->insts_d, ctx->romwork_d, ctx->nromwork, ctx->run_d,
                                       par, 0, ctx->groups_d, ctx->gwork_d, ctx->ngwork, ctx->ginst_d);
    CK(cudaEventRecord(e[2], ctx->stream));
    advance_kernel<<<1, 32, 0, ctx->stream>>>(ctx->run_d, 1);
    CK(cudaGetLastError());
    ctx->n_yee += 1;
    ctx->n_post += post ? 1 : 0;
    ctx->ev_used += 3;
    if (ctx->ev_used == (int)ctx->ev.size()) {
      int rc = drain_events(ctx);
      if (rc) return rc;
    }
  }
  ctx->cur ^= (int)(nsteps & 1);
  ctx->step += nsteps;
  return FDTD_OK;
}

// The zone chain of one pair of steps on the side stream (highest priority,
// so that its blocks are scheduled ahead of the march's pending ones),
// forked from and joined back into s: half 0, map, half 1, map.
// Device tables of a two-step launch: the context's own, or the gradient
// recomputation's per-pair tables (frames of E and the model states).
struct TbTables {
  const SimDev* sims;
  const RomInstDev* insts;
  const RunDev* run;
  MarchFn march;
};

TbTables own_tables(const fdtd_ctx* ctx) {
  return {ctx->sims_d, ctx->insts_d, ctx->run_d, ctx->tb_march ? march_fn(ctx->tbm_mb, ctx->tbm_ring, ctx->tbm_sparse)
                                                               : nullptr};
}

void launch_chain(fdtd_ctx* ctx, cudaStream_t s, int par, int c, const TbTables& tt) {
  const unsigned nz = (unsigned)ctx->tb_nchain;
  const TbTile* zt = ctx->tb_tiles_d + (ctx->tb_tiles.size() - nz);
  cudaStream_t q = ctx->side_stream;
  cudaEventRecord(ctx->ev_fork, s);
  cudaStreamWaitEvent(q, ctx->ev_fork, 0);
  const unsigned nmap = (unsigned)(ctx->chain_nrow + ctx->ngwork);
  launch_k(zone_step_kernel<0>, nz, kTbThreads, ctx->zone_smem, q, false, ctx->prio_hi, tt.sims, zt, tt.insts, tt.run,
           (const TbRun*)ctx->tb_run_d, ctx->zone_scratch.p, par, c);
  launch_k(rom_chain_kernel, nmap, kRomRowsPerCta * 32, ctx->chain_smem, q, false, ctx->prio_hi, tt.sims, tt.insts,
           (const RomWork*)ctx->romwork_d, ctx->chain_nrow, (const GemmGroupDev*)ctx->groups_d,
           (const GemmWork*)ctx->gwork_d, (const int*)ctx->ginst_d, par, 0);
  launch_k(zone_step_kernel<1>, nz, kTbThreads, ctx->zone_smem, q, false, ctx->prio_hi, tt.sims, zt, tt.insts, tt.run,
           (const TbRun*)ctx->tb_run_d, ctx->zone_scratch.p, par, c);
  launch_k(rom_chain_kernel, nmap, kRomRowsPerCta * 32, ctx->chain_smem, q, false, ctx->prio_hi, tt.sims, tt.insts,
           (const RomWork*)ctx->romwork_d, ctx->chain_nrow, (const GemmGroupDev*)ctx->groups_d,
           (const GemmWork*)ctx->gwork_d, (const int*)ctx->ginst_d, par, 1);
  cudaEventRecord(ctx->ev_join, q);
}

void launch_tb(fdtd_ctx* ctx, cudaStream_t s, int par, int c, const TbTables& tt) {
  const unsigned ntb = (unsigned)(ctx->tb_tiles.size() - ctx->tb_nchain);   // ordinary and fused model tiles
  if (ctx->tb_nchain > 0) launch_chain(ctx, s, par, c, tt);
  if (ntb > 0)
    yee_tb2_kernel<<<ntb, kTbThreads, kTbSmemFields, s>>>(tt.sims, ctx->tb_tiles_d, tt.insts, tt.run, ctx->tb_run_d,
                                                          par, c);
  if (ctx->tb_march)   // overlaps the model tiles (programmatic serialisation) when there are any
    launch_k(tt.march, (unsigned)ctx->tbm_tiles.size(), 32 * ctx->tbm_w, march_smem(ctx->tbm_ring, ctx->tbm_w), s,
             ctx->pdl && ntb > 0,
             tt.sims, (const TileWork*)ctx->tbm_tiles_d, tt.run, (const TbMarchDev*)ctx->tbm_d, par, c, ctx->tbm_pf);
  if (ctx->tb_nchain > 0) cudaStreamWaitEvent(s, ctx->ev_join, 0);
}

void launch_tb(fdtd_ctx* ctx, cudaStream_t s, int par, int c) { launch_tb(ctx, s, par, c, own_tables(ctx)); }

int ensure_tb_graph(fdtd_ctx* ctx, int par, int nprobe) {
  if (ctx->tb_graph[par] && ctx->tb_graph_nprobe[par] == nprobe) return FDTD_OK;
  if (ctx->tb_graph[par]) cudaGraphExecDestroy(ctx->tb_graph[par]);
  ctx->tb_graph[par] = nullptr;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
  for (int c = 0; c < kChunk / 2; ++c) launch_tb(ctx, ctx->capture_stream, par ^ (c & 1), c);
  advance_kernel<<<1, 32, 0, ctx->capture_stream>>>(ctx->run_d, kChunk);
  CK(cudaStreamEndCapture(ctx->capture_stream, &g));
  cudaError_t e = cudaGraphInstantiate(&ctx->tb_graph[par], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, FDTD_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  ctx->tb_graph_nprobe[par] = nprobe;
  return FDTD_OK;
}

// Two steps per launch: graph replays of kChunk steps, then pairs, then (odd
// counts) one step of the one-step kernels.
int march_tb(fdtd_ctx* ctx, long long nsteps, int nprobe) {
  const int nprobe_blocks = post_extra_blocks(ctx, nprobe);
  long long done = 0;
  if (nsteps >= kChunk) {
    int rc = ensure_tb_graph(ctx, ctx->cur, nprobe);
    if (rc) return rc;
    for (; done + kChunk <= nsteps; done += kChunk) CK(cudaGraphLaunch(ctx->tb_graph[ctx->cur], ctx->stream));
  }
  const int rem = (int)(nsteps - done);
  int par = ctx->cur;
  for (int c = 0; c < rem / 2; ++c, par ^= 1) launch_tb(ctx, ctx->stream, par, c);
  if (rem & 1) {
    launch_step(ctx, ctx->stream, par, 2 * (rem / 2), nprobe_blocks);
    par ^= 1;
  }
  CK(cudaGetLastError());
  ctx->cur = par;
  ctx->step += nsteps;
  return FDTD_OK;
}

int march(fdtd_ctx* ctx, long long nsteps, int nprobe) {
  if (ctx->timing) return march_timed(ctx, nsteps, nprobe);
  if (ctx->tb && ctx->dft_nmon == 0) return march_tb(ctx, nsteps, nprobe);
  const int nprobe_blocks = post_extra_blocks(ctx, nprobe);
  long long done = 0;
  if (nsteps >= kChunk) {
    int rc = ensure_graph(ctx, ctx->cur, nprobe_blocks);
    if (rc) return rc;
    for (; done + kChunk <= nsteps; done += kChunk) CK(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
  }
  const int rem = (int)(nsteps - done);
  for (int c = 0; c < rem; ++c) launch_step(ctx, ctx->stream, ctx->cur ^ (c & 1), c, nprobe_blocks);
  CK(cudaGetLastError());
  ctx->cur ^= (rem & 1);
  ctx->step += nsteps;
  return FDTD_OK;
}

}  // namespace

namespace {

// Tile height th minimising ceil(T / slots) * (th + 1) over 8..128 rows
// (T = tiles of kCtaCols columns x th rows over every simulation).
int best_tile_rows(const std::vector<SimHost>& sims, long long slots) {
  auto total = [&](int th) {
    long long t = 0;
    for (const SimHost& sh : sims) t += (long long)((sh.nx + kCtaCols - 1) / kCtaCols) * ((sh.ny + th - 1) / th);
    return t;
  };
  int best = 32;
  long long best_cost = -1;
  for (int th = 8; th <= 128; ++th) {
    const long long cost = ((total(th) + slots - 1) / slots) * (th + 1);
    if (best_cost < 0 || cost <= best_cost) best_cost = cost, best = th;
  }
  return best;
}

// Tile table of kCtaCols x th tiles over every simulation.
std::vector<TileWork> tile_table(const std::vector<SimHost>& sims, int th) {
  std::vector<TileWork> t;
  for (int s = 0; s < (int)sims.size(); ++s) {
    const SimHost& sh = sims[s];
    for (int ty = 0; ty < (sh.ny + th - 1) / th; ++ty)
      for (int tx = 0; tx < (sh.nx + kCtaCols - 1) / kCtaCols; ++tx)
        t.push_back({s, tx * kCtaCols, ty * th, std::min(sh.ny, (ty + 1) * th)});
  }
  return t;
}

// Tile plan of the stencil kernel.  A CTA covers kCtaCols columns; the tile
// height th (same for every simulation) is chosen so that the tiles fill
// whole waves of resident CTAs: minimise ceil(T / slots) * (th + 1) (the +1
// is the recomputed halo row), T = total tiles, slots = SMs x resident CTAs.
// FDTD_VEC (2 or 4) and FDTD_TILE_ROWS override the choice (results are
// identical; only speed changes).
void plan_tiles(fdtd_ctx* ctx) {
  ctx->run_sig.clear();
  int vec = 4;
  if (const char* e = getenv("FDTD_VEC")) vec = (atoi(e) == 2) ? 2 : 4;
  ctx->vec = vec;
  ctx->stencil_tma = false;
  if (const char* e = getenv("FDTD_STENCIL")) ctx->stencil_tma = (vec == 4) && std::string(e) == "tma";
  ctx->pdl = true;
  if (const char* e = getenv("FDTD_PDL")) ctx->pdl = atoi(e) != 0;
  ctx->pf1 = 0;
  if (const char* e = getenv("FDTD_PF1")) ctx->pf1 = std::min(8, std::max(0, atoi(e)));
  int dev = 0, nsm = 1, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (ctx->stencil_tma)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, yee_step_tma_kernel, kCtaCols / 4, kTmaSmem);
  else if (vec == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, yee_step_kernel<2>, kCtaCols / 2, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, yee_step_kernel<4>, kCtaCols / 4, 0);
  const long long slots = (long long)nsm * std::max(occ, 1);
  int best = best_tile_rows(ctx->sims, slots);
  if (const char* e = getenv("FDTD_TILE_ROWS"))
    best = std::min(512, std::max(4, atoi(e)));   // <= 512: one warp's 32 bit words cover a tile
  if (ctx->ov_th1) best = ctx->ov_th1;
  ctx->tiles.clear();
  for (int s = 0; s < (int)ctx->sims.size(); ++s) {
    SimHost& sh = ctx->sims[s];
    sh.th = best;
    sh.ncx = (sh.nx + kCtaCols - 1) / kCtaCols;
    sh.ncy = (sh.ny + best - 1) / best;
    sh.tile_base = (int)ctx->tiles.size();
    for (int ty = 0; ty < sh.ncy; ++ty)
      for (int tx = 0; tx < sh.ncx; ++tx)
        ctx->tiles.push_back({s, tx * kCtaCols, ty * best, std::min(sh.ny, (ty + 1) * best)});
  }
}

// Fixed device array used by fdtd_energy_noalloc for its partial sums.  In
// host code its name is only a stand-in: the device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// cached.
__device__ __align__(256) double g_energy_static[FDTD_ENERGY_STATIC_MAX];

int static_energy_scratch(fdtd_ctx* ctx, double** ptr) {
  static std::mutex mu;
  static std::vector<void*> addr;   // per device ordinal
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_energy_static));
    addr[dev] = p;
  }
  *ptr = static_cast<double*>(addr[dev]);
  return FDTD_OK;
}

}  // namespace

#include "adjoint.cuh"
#include "tune.cuh"

// ============================================================== C ABI

extern "C" {

const char* fdtd_last_error(const fdtd_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_err;
  return copy.c_str();
}

int fdtd_cfl_limit(double dx, double dy, double* out) {
  if (!(dx > 0) || !(dy > 0) || !out) return set_global_error(FDTD_EINVAL, "fdtd_cfl_limit: bad argument");
  const double c0 = 1.0 / std::sqrt(kEps0 * kMu0);
  *out = 1.0 / (c0 * std::sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy)));
  return FDTD_OK;
}

void fdtd_destroy(fdtd_ctx* ctx) {
  if (!ctx) return;
  drop_graphs(ctx);
  for (SimHost& s : ctx->sims) {
    for (int p = 0; p < 2; ++p) {
      cudaFree(s.ex[p]);
      cudaFree(s.ey[p]);
      cudaFree(s.hz[p]);
    }
    cudaFree(s.mat_d);
    cudaFree(s.mbits_d);
  }
  for (Instance& in : ctx->insts) {
    for (float* p : in.state_d) cudaFree(p);
    cudaFree(in.y_edge_d);
    cudaFree(in.h_cell_d);
  }
  ctx->insts.clear();   // releases the shared maps
  cudaFree(ctx->sims_d);
  cudaFree(ctx->tiles_d);
  cudaFree(ctx->insts_d);
  cudaFree(ctx->romwork_d);
  cudaFree(ctx->groups_d);
  cudaFree(ctx->gwork_d);
  cudaFree(ctx->ginst_d);
  cudaFree(ctx->tb_tiles_d);
  cudaFree(ctx->tb_zones_d);
  cudaFree(ctx->tb_run_d);
  ctx->tb_src.release();
  ctx->tb_prb.release();
  cudaFree(ctx->tbm_tiles_d);
  cudaFree(ctx->tbm_zone_rng_d);
  cudaFree(ctx->tbm_zones_d);
  cudaFree(ctx->tbm_d);
  ctx->tbm_src_rng.release();
  ctx->tbm_ent_sim.release();
  ctx->tbm_prb_rng.release();
  ctx->tbm_src.release();
  ctx->tbm_prb.release();
  cudaFree(ctx->run_d);
  for (fdtd_ctx::RunSlot& sl : ctx->run_slots) {
    if (sl.done) {
      cudaEventSynchronize(sl.done);
      cudaEventDestroy(sl.done);
    }
    if (sl.host) cudaFreeHost(sl.host);
  }
  cudaFree(ctx->status_d);
  cudaFree(ctx->einst_d);
  cudaFree(ctx->tile_base_d);
  ctx->energy_scratch.release();
  ctx->src_range.release();
  ctx->src_edges.release();
  ctx->waves.release();
  ctx->probe_sim.release();
  ctx->probe_cell.release();
  ctx->host_waves.release();
  ctx->host_probes.release();
  ctx->pml_coef_d.release();
  ctx->pml_sims_d.release();
  ctx->pml_cells_d.release();
  ctx->pml_edges_d.release();
  ctx->pml_psi.release();
  ctx->dft_sim.release();
  ctx->dft_cell.release();
  ctx->dft_fdt.release();
  ctx->dft_acc.release();
  for (auto& b : ctx->bases) {
    cudaFree(b.V1);
    cudaFree(b.V2);
  }
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  ctx->zone_scratch.release();
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
}

int fdtd_create(const fdtd_grid_desc* g, void* cuda_stream, fdtd_ctx** out) {
  fdtd_ctx* ctx = nullptr;
  if (!g || !out || g->nsim < 1 || !g->sims) return fail(ctx, FDTD_EINVAL, "fdtd_create: null or empty descriptor");
  if (!(g->dx > 0) || !(g->dy > 0) || !(g->dt > 0)) return fail(ctx, FDTD_EINVAL, "fdtd_create: dx, dy, dt must be > 0");
  double lim;
  fdtd_cfl_limit(g->dx, g->dy, &lim);
  if (!(g->dt < lim)) return fail(ctx, FDTD_ECFL, "fdtd_create: dt is not below the coarse CFL limit (Eq. (1))");
  for (int s = 0; s < g->nsim; ++s) {
    const fdtd_sim_desc& sd = g->sims[s];
    if (sd.nx < 2 || sd.ny < 2 || !sd.eps_r || !sd.sigma)
      return fail(ctx, FDTD_EINVAL, "fdtd_create: simulation " + std::to_string(s) + " malformed");
    if ((long long)(sd.ny + 1) * (((sd.nx + 1 + 127) / 128) * 128) >= (1ll << 30))
      return fail(ctx, FDTD_EINVAL, "fdtd_create: grid too large (2^30 floats per field)");
    for (long long k = 0; k < (long long)sd.nx * sd.ny; ++k)
      if (!(sd.eps_r[k] > 0) || !(sd.sigma[k] >= 0))
        return fail(ctx, FDTD_EINVAL, "fdtd_create: eps_r must be > 0 and sigma >= 0");
  }
  ctx = new (std::nothrow) fdtd_ctx();
  if (!ctx) return set_global_error(FDTD_ENOMEM, "fdtd_create: out of host memory");
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->dx = g->dx, ctx->dy = g->dy, ctx->dt = g->dt;
  auto bail = [&](int code) {
    std::string m = ctx->err;
    fdtd_destroy(ctx);
    set_global_error(code, m);
    return code;
  };
  if (cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->err = "fdtd_create: cannot create a CUDA stream";
    return bail(FDTD_ECUDA);
  }
  ctx->sims.resize(g->nsim);
  std::vector<SimDev> sdev(g->nsim);
  for (int s = 0; s < g->nsim; ++s) {
    const fdtd_sim_desc& d = g->sims[s];
    SimHost& sh = ctx->sims[s];
    sh.nx = d.nx, sh.ny = d.ny;
    sh.pitch = ((d.nx + 1 + 127) / 128) * 128;
    const size_t ncell = (size_t)d.nx * d.ny;
    sh.eps_r.assign(d.eps_r, d.eps_r + ncell);
    sh.sigma.assign(d.sigma, d.sigma + ncell);
    sh.region.assign(ncell, 0);
    sh.mat.assign((size_t)(d.ny + 1) * sh.pitch, make_float2(0.f, 0.f));
    for (int j = 0; j < d.ny; ++j)
      for (int i = 0; i < d.nx; ++i) {
        const size_t k = (size_t)j * d.nx + i;
        sh.mat[(size_t)j * sh.pitch + i] =
            make_float2((float)(kEps0 * d.eps_r[k] / g->dt + 0.5 * d.sigma[k]), (float)d.sigma[k]);
      }
    const size_t bytes = sizeof(float) * (size_t)(d.ny + 1) * sh.pitch;
    for (int p = 0; p < 2; ++p) {
      if (cudaMalloc(&sh.ex[p], bytes) != cudaSuccess || cudaMalloc(&sh.ey[p], bytes) != cudaSuccess ||
          cudaMalloc(&sh.hz[p], bytes) != cudaSuccess) {
        ctx->err = "fdtd_create: device allocation failed";
        return bail(FDTD_ENOMEM);
      }
      cudaMemset(sh.ex[p], 0, bytes);
      cudaMemset(sh.ey[p], 0, bytes);
      cudaMemset(sh.hz[p], 0, bytes);
    }
    sh.nstrip = sh.pitch / 128;
    const char* md = getenv("FDTD_MAT_DENSE");
    sh.all_dense = (md && atoi(md) == 1) || !pick_background(sh, &sh.mbg);
    sh.mbits.assign((size_t)((d.ny + 31) / 32) * sh.nstrip, 0u);
    update_mbits(sh, 0, d.ny);
    if (cudaMalloc(&sh.mat_d, sizeof(float2) * sh.mat.size()) != cudaSuccess ||
        cudaMalloc(&sh.mbits_d, sizeof(uint32_t) * sh.mbits.size()) != cudaSuccess) {
      ctx->err = "fdtd_create: device allocation failed";
      return bail(FDTD_ENOMEM);
    }
    cudaMemcpy(sh.mat_d, sh.mat.data(), sizeof(float2) * sh.mat.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(sh.mbits_d, sh.mbits.data(), sizeof(uint32_t) * sh.mbits.size(), cudaMemcpyHostToDevice);
    SimDev& sd = sdev[s];
    for (int p = 0; p < 2; ++p) sd.ex[p] = sh.ex[p], sd.ey[p] = sh.ey[p], sd.hz[p] = sh.hz[p];
    sd.mat = sh.mat_d;
    sd.mbits = sh.mbits_d;
    sd.mbg = sh.mbg;
    sd.nstrip = sh.nstrip;
    sd.nx = d.nx, sd.ny = d.ny, sd.pitch = sh.pitch;
    sd.chx = (float)(g->dt / (kMu0 * g->dy));
    sd.chy = (float)(g->dt / (kMu0 * g->dx));
    sd.rdy = (float)(1.0 / g->dy);
    sd.rdx = (float)(1.0 / g->dx);
    sd.rdy2 = 2.f * sd.rdy;   // exact
    sd.rdx2 = 2.f * sd.rdx;
  }
  plan_tiles(ctx);
  if (const char* e = getenv("FDTD_TB")) ctx->tb_mode = atoi(e) != 0 ? 1 : 0;   // fixed for the context
  if (const char* e = getenv("FDTD_TB_CHAIN")) ctx->tb_chain_mode = atoi(e) == 0 ? 0 : atoi(e) == 2 ? -1 : 1;
  if (plan_tb(ctx) != FDTD_OK) return bail(FDTD_ECUDA);
  if (cudaMalloc(&ctx->sims_d, sizeof(SimDev) * sdev.size()) != cudaSuccess ||
      cudaMalloc(&ctx->tiles_d, sizeof(TileWork) * ctx->tiles.size()) != cudaSuccess ||
      cudaMalloc(&ctx->run_d, sizeof(RunDev)) != cudaSuccess ||
      cudaMalloc(&ctx->status_d, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ctx->status_d, 0, sizeof(unsigned)) != cudaSuccess) {
    ctx->err = "fdtd_create: device allocation failed";
    return bail(FDTD_ENOMEM);
  }
  cudaMemcpy(ctx->sims_d, sdev.data(), sizeof(SimDev) * sdev.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(ctx->tiles_d, ctx->tiles.data(), sizeof(TileWork) * ctx->tiles.size(), cudaMemcpyHostToDevice);
  {
    std::vector<int> tb(g->nsim + 1);
    for (int s = 0; s < g->nsim; ++s) tb[s] = ctx->sims[s].tile_base;
    tb[g->nsim] = (int)ctx->tiles.size();
    if (cudaMalloc(&ctx->tile_base_d, sizeof(int) * tb.size()) != cudaSuccess) {
      ctx->err = "fdtd_create: device allocation failed";
      return bail(FDTD_ENOMEM);
    }
    cudaMemcpy(ctx->tile_base_d, tb.data(), sizeof(int) * tb.size(), cudaMemcpyHostToDevice);
  }
  cudaMemset(ctx->run_d, 0, sizeof(RunDev));
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ctx->err = std::string("fdtd_create: ") + cudaGetErrorString(e);
    return bail(FDTD_ECUDA);
  }
  *out = ctx;
  return FDTD_OK;
}

int rom_embed(fdtd_ctx* ctx, const rom_model* m, int sim, int i0, int j0, int* inst_out) {
  NvtxRange nvtx_("rom_embed");
  if (!ctx || !m) return fail(ctx, FDTD_EINVAL, "rom_embed: null argument");
  if (sim < 0 || sim >= (int)ctx->sims.size()) return fail(ctx, FDTD_EINVAL, "rom_embed: sim out of range");
  if (std::fabs(m->dt - ctx->dt) > 1e-12 * ctx->dt || std::fabs(m->dx - ctx->dx) > 1e-12 * ctx->dx ||
      std::fabs(m->dy - ctx->dy) > 1e-12 * ctx->dy)
    return fail(ctx, FDTD_EINVAL, "rom_embed: model built for another dx, dy or dt");
  SimHost& sh = ctx->sims[sim];
  const int a = m->a, b = m->b;
  if (i0 < 1 || j0 < 1 || i0 + a > sh.nx - 1 || j0 + b > sh.ny - 1)
    return fail(ctx, FDTD_EINVAL, "rom_embed: region must keep one coarse cell from the walls");
  for (int j = j0 - 1; j <= j0 + b; ++j)
    for (int i = i0 - 1; i <= i0 + a; ++i)
      if (sh.region[(size_t)j * sh.nx + i])
        return fail(ctx, FDTD_EINVAL, "rom_embed: region overlaps or touches another region");
  for (int j = j0 - 2; j < j0 + b + 2; ++j)
    for (int i = i0 - 2; i < i0 + a + 2; ++i)
      if (pml_cell(ctx, sim, i, j))
        return fail(ctx, FDTD_EINVAL, "rom_embed: region within two cells of a PML layer");
  Instance in;
  in.sim = sim, in.i0 = i0, in.j0 = j0, in.a = a, in.b = b, in.q = m->qE + m->qH;
  in.itf = make_interface(i0, j0, a, b, ctx->dx, ctx->dy, ctx->dt, sh.eps_r.data(), sh.sigma.data(), sh.nx);
  in.ny = in.itf.ny;
  in.n = in.ny + in.q;
  std::vector<double> key(in.itf.dplus);
  key.insert(key.end(), in.itf.dminus.begin(), in.itf.dminus.end());
  key.insert(key.end(), in.itf.dlg.begin(), in.itf.dlg.end());
  for (const Instance& o : ctx->insts)
    if (o.map->model_id == m->id && o.map->key == key) {
      in.map = o.map;
      break;
    }
  if (!in.map) {
    auto cm = std::make_shared<CoupledMap>();
    cm->model_id = m->id;
    cm->key = key;
    std::string msg;
    int rc = couple(*m, in.itf, ctx->dt, cm->P, cm->Q, msg);
    if (rc) return fail(ctx, rc, "rom_embed: " + msg);
    // [P | Q] in FP32, rows padded to a multiple of 4 floats (16-B aligned).
    cm->ld = ((in.n + in.ny + 3) / 4) * 4;
    std::vector<float> Mf((size_t)in.n * cm->ld, 0.f);
    for (int r = 0; r < in.n; ++r) {
      for (int k = 0; k < in.n; ++k) Mf[(size_t)r * cm->ld + k] = (float)cm->P(r, k);
      for (int k = 0; k < in.ny; ++k) Mf[(size_t)r * cm->ld + in.n + k] = (float)cm->Q(r, k);
    }
    CK(cudaMalloc(&cm->M_d, sizeof(float) * Mf.size()));
    CK(cudaMemcpy(cm->M_d, Mf.data(), sizeof(float) * Mf.size(), cudaMemcpyHostToDevice));
    // storage-function data: R~ at the run dt (Eq. (12)) and the half cells
    const int q = in.q, qE = m->qE, qH = m->qH;
    std::vector<double> R((size_t)q * q, 0.0), cc(2 * (size_t)in.ny);
    for (int i = 0; i < qE; ++i)
      for (int j = 0; j < qE; ++j) R[(size_t)i * q + j] = m->R11(i, j) / ctx->dt;
    for (int i = 0; i < qH; ++i)
      for (int j = 0; j < qH; ++j) R[(size_t)(qE + i) * q + qE + j] = m->R22(i, j) / ctx->dt;
    for (int i = 0; i < qE; ++i)
      for (int j = 0; j < qH; ++j) R[(size_t)i * q + qE + j] = R[(size_t)(qE + j) * q + i] = -0.5 * m->Kt(i, j);
    for (int k = 0; k < in.ny; ++k) {
      // dplus = Dl Dl' (eps_b/dt + sig_b/2), dminus = Dl Dl' (eps_b/dt - sig_b/2)
      cc[k] = 0.25 * (in.itf.dplus[k] + in.itf.dminus[k]) * ctx->dt;   // 1/2 Dl Dl' eps_b
      cc[in.ny + k] = 0.5 * ctx->dt * in.itf.dlg[k];
    }
    CK(cudaMalloc(&cm->R_d, sizeof(double) * R.size()));
    CK(cudaMalloc(&cm->c_d, sizeof(double) * cc.size()));
    CK(cudaMemcpy(cm->R_d, R.data(), sizeof(double) * R.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(cm->c_d, cc.data(), sizeof(double) * cc.size(), cudaMemcpyHostToDevice));
    in.map = cm;
  }
  for (int k = 0; k < in.ny; ++k) {
    in.y_edge.push_back((in.itf.comp[k] << 30) | (in.itf.ej[k] * sh.pitch + in.itf.ei[k]));
    in.h_cell.push_back(in.itf.hj[k] * sh.pitch + in.itf.hi[k]);
  }
  // [y; x~] padded to ld floats: the two-step path's maps outside the tile
  // read the whole input vector [y; x~; h; 0] from it (the padding stays 0)
  for (int p = 0; p < 3; ++p) {
    CK(cudaMalloc(&in.state_d[p], sizeof(float) * in.map->ld));
    CK(cudaMemset(in.state_d[p], 0, sizeof(float) * in.map->ld));
  }
  CK(cudaMalloc(&in.y_edge_d, sizeof(int) * in.ny));
  CK(cudaMalloc(&in.h_cell_d, sizeof(int) * in.ny));
  CK(cudaMemcpy(in.y_edge_d, in.y_edge.data(), sizeof(int) * in.ny, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(in.h_cell_d, in.h_cell.data(), sizeof(int) * in.ny, cudaMemcpyHostToDevice));
  // Mark the covered cells and zero every field on and inside the region.
  CK(cudaStreamSynchronize(ctx->stream));
  for (int j = j0; j < j0 + b; ++j)
    for (int i = i0; i < i0 + a; ++i) {
      sh.region[(size_t)j * sh.nx + i] = 1;
      sh.mat[(size_t)j * sh.pitch + i].x = -1.f;
    }
  update_mbits(sh, j0, j0 + b);
  CK(cudaMemcpy(sh.mat_d, sh.mat.data(), sizeof(float2) * sh.mat.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sh.mbits_d, sh.mbits.data(), sizeof(uint32_t) * sh.mbits.size(), cudaMemcpyHostToDevice));
  for (int p = 0; p < 2; ++p) {
    for (int j = j0; j <= j0 + b; ++j) {
      CK(cudaMemset(sh.ex[p] + (size_t)j * sh.pitch + i0, 0, sizeof(float) * a));
      if (j < j0 + b) {
        CK(cudaMemset(sh.ey[p] + (size_t)j * sh.pitch + i0, 0, sizeof(float) * (a + 1)));
        CK(cudaMemset(sh.hz[p] + (size_t)j * sh.pitch + i0, 0, sizeof(float) * a));
      }
    }
  }
  ctx->insts.push_back(std::move(in));
  int rc = upload_instances(ctx);
  if (rc) return rc;
  if (inst_out) *inst_out = (int)ctx->insts.size() - 1;
  return FDTD_OK;
}

int fdtd_get_rom_map(const fdtd_ctx* ctx, int inst, int* n, int* ny, double* P, double* Q) {
  if (!ctx || inst < 0 || inst >= (int)ctx->insts.size())
    return set_global_error(FDTD_EINVAL, "fdtd_get_rom_map: bad instance");
  const Instance& in = ctx->insts[inst];
  if (n) *n = in.n;
  if (ny) *ny = in.ny;
  if (P) std::memcpy(P, in.map->P.a.data(), sizeof(double) * in.map->P.a.size());
  if (Q) std::memcpy(Q, in.map->Q.a.data(), sizeof(double) * in.map->Q.a.size());
  return FDTD_OK;
}

// The sources' positions (waveforms dropped) and the probes of a run.
static void remember_layout(fdtd_ctx* ctx, const fdtd_source* src, int nsrc, const fdtd_probe* probes, int nprobe) {
  ctx->last_src.assign(src, src + nsrc);
  for (fdtd_source& s : ctx->last_src) s.wave = nullptr;
  ctx->last_prb.assign(probes, probes + nprobe);
}

int fdtd_run(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
             const fdtd_probe* probes, int nprobe, float* probe_out) {
  NvtxRange nvtx_("fdtd_run");
  if (!ctx || nsteps < 0 || nsrc < 0 || nprobe < 0 || (nsrc && !src) || (nprobe && !probes))
    return fail(ctx, FDTD_EINVAL, "fdtd_run: bad argument");
  if (nsteps == 0) return FDTD_OK;
  std::vector<const float*> w(std::max(nsrc, 1));
  for (int s = 0; s < nsrc; ++s) w[s] = src[s].wave;
  int rc = prepare_run(ctx, nsteps, src, nsrc, w.data(), probes, nprobe, probe_out);
  if (rc) return rc;
  remember_layout(ctx, src, nsrc, probes, nprobe);
  return march(ctx, nsteps, nprobe);
}

int fdtd_run_host(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
                  const fdtd_probe* probes, int nprobe, float* probe_out_host) {
  NvtxRange nvtx_("fdtd_run_host");
  if (!ctx || nsteps < 0 || nsrc < 0 || nprobe < 0 || (nsrc && !src) || (nprobe && !probes) ||
      (nprobe && !probe_out_host))
    return fail(ctx, FDTD_EINVAL, "fdtd_run_host: bad argument");
  if (nsteps == 0) return FDTD_OK;
  for (int s = 0; s < nsrc; ++s)
    if (!src[s].wave) return fail(ctx, FDTD_EINVAL, "fdtd_run_host: null waveform");
  CK(ctx->host_waves.reserve((size_t)std::max(nsrc, 1) * nsteps));
  CK(ctx->host_probes.reserve((size_t)std::max(nprobe, 1) * nsteps));
  std::vector<const float*> w(std::max(nsrc, 1));
  for (int s = 0; s < nsrc; ++s) {
    w[s] = ctx->host_waves.p + (size_t)s * nsteps;
    CK(cudaMemcpyAsync((void*)w[s], src[s].wave, sizeof(float) * nsteps, cudaMemcpyHostToDevice, ctx->stream));
  }
  int rc = prepare_run(ctx, nsteps, src, nsrc, w.data(), probes, nprobe, ctx->host_probes.p);
  if (rc) return rc;
  remember_layout(ctx, src, nsrc, probes, nprobe);
  rc = march(ctx, nsteps, nprobe);
  if (rc) return rc;
  if (nprobe > 0)
    CK(cudaMemcpyAsync(probe_out_host, ctx->host_probes.p, sizeof(float) * nsteps * nprobe,
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  rc = check_status(ctx);
  if (rc) return rc;
  for (long long k = 0; k < nsteps * nprobe; ++k)
    if (!std::isfinite(probe_out_host[k]))
      return fail(ctx, FDTD_EUNSTABLE, "fdtd_run_host: non-finite probe sample at step " + std::to_string(k / nprobe));
  return FDTD_OK;
}

int fdtd_get_fields(fdtd_ctx* ctx, int sim, float* Ex, float* Ey, float* Hz) {
  if (!ctx || sim < 0 || sim >= (int)ctx->sims.size()) return fail(ctx, FDTD_EINVAL, "fdtd_get_fields: bad sim");
  const SimHost& sh = ctx->sims[sim];
  const int c = ctx->cur;
  const size_t sp = sizeof(float) * sh.pitch;
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);
  if (rc) return rc;
  if (Ex) CK(cudaMemcpy2D(Ex, sizeof(float) * sh.nx, sh.ex[c], sp, sizeof(float) * sh.nx, sh.ny + 1, cudaMemcpyDeviceToHost));
  if (Ey) CK(cudaMemcpy2D(Ey, sizeof(float) * (sh.nx + 1), sh.ey[c], sp, sizeof(float) * (sh.nx + 1), sh.ny, cudaMemcpyDeviceToHost));
  if (Hz) CK(cudaMemcpy2D(Hz, sizeof(float) * sh.nx, sh.hz[c], sp, sizeof(float) * sh.nx, sh.ny, cudaMemcpyDeviceToHost));
  return FDTD_OK;
}

int fdtd_set_fields(fdtd_ctx* ctx, int sim, const float* Ex, const float* Ey, const float* Hz) {
  if (!ctx || sim < 0 || sim >= (int)ctx->sims.size() || !Ex || !Ey || !Hz)
    return fail(ctx, FDTD_EINVAL, "fdtd_set_fields: bad argument");
  const SimHost& sh = ctx->sims[sim];
  const int nx = sh.nx, ny = sh.ny;
  // Clean copies: PEC walls and covered cells/edges held at 0.
  std::vector<float> ex((size_t)(ny + 1) * nx, 0.f), ey((size_t)ny * (nx + 1), 0.f), hz((size_t)ny * nx, 0.f);
  auto reg = [&](int i, int j) { return sh.region[(size_t)j * nx + i] != 0; };
  for (int j = 1; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (!(reg(i, j - 1) && reg(i, j))) ex[(size_t)j * nx + i] = Ex[(size_t)j * nx + i];
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i)
      if (!(reg(i - 1, j) && reg(i, j))) ey[(size_t)j * (nx + 1) + i] = Ey[(size_t)j * (nx + 1) + i];
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (!reg(i, j)) hz[(size_t)j * nx + i] = Hz[(size_t)j * nx + i];
  const size_t dp = sizeof(float) * sh.pitch;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int p = 0; p < 2; ++p) {
    CK(cudaMemcpy2D(sh.ex[p], dp, ex.data(), sizeof(float) * nx, sizeof(float) * nx, ny + 1, cudaMemcpyHostToDevice));
    CK(cudaMemcpy2D(sh.ey[p], dp, ey.data(), sizeof(float) * (nx + 1), sizeof(float) * (nx + 1), ny, cudaMemcpyHostToDevice));
    CK(cudaMemcpy2D(sh.hz[p], dp, hz.data(), sizeof(float) * nx, sizeof(float) * nx, ny, cudaMemcpyHostToDevice));
  }
  // Interface values become each model's y.
  for (Instance& in : ctx->insts) {
    if (in.sim != sim) continue;
    std::vector<float> y(in.ny);
    for (int k = 0; k < in.ny; ++k)
      y[k] = in.itf.comp[k] == 0 ? ex[(size_t)in.itf.ej[k] * nx + in.itf.ei[k]]
                                 : ey[(size_t)in.itf.ej[k] * (nx + 1) + in.itf.ei[k]];
    for (int p = 0; p < 2; ++p) CK(cudaMemcpy(in.state_d[p], y.data(), sizeof(float) * in.ny, cudaMemcpyHostToDevice));
  }
  return FDTD_OK;
}

int fdtd_get_rom_state(fdtd_ctx* ctx, int inst, float* x) {
  if (!ctx || inst < 0 || inst >= (int)ctx->insts.size() || !x) return fail(ctx, FDTD_EINVAL, "fdtd_get_rom_state: bad argument");
  const Instance& in = ctx->insts[inst];
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(x, in.state_d[ctx->cur] + in.ny, sizeof(float) * in.q, cudaMemcpyDeviceToHost));
  return FDTD_OK;
}

int fdtd_set_rom_state(fdtd_ctx* ctx, int inst, const float* x) {
  if (!ctx || inst < 0 || inst >= (int)ctx->insts.size() || !x) return fail(ctx, FDTD_EINVAL, "fdtd_set_rom_state: bad argument");
  const Instance& in = ctx->insts[inst];
  CK(cudaStreamSynchronize(ctx->stream));
  for (int p = 0; p < 2; ++p) CK(cudaMemcpy(in.state_d[p] + in.ny, x, sizeof(float) * in.q, cudaMemcpyHostToDevice));
  return FDTD_OK;
}

int fdtd_energy(fdtd_ctx* ctx, double* out) {
  NvtxRange nvtx_("fdtd_energy");
  if (!ctx || !out) return fail(ctx, FDTD_EINVAL, "fdtd_energy: bad argument");
  const int ntiles = (int)ctx->tiles.size(), ninst = (int)ctx->insts.size();
  const int nsim = (int)ctx->sims.size();
  CK(ctx->energy_scratch.reserve((size_t)ntiles + ninst + nsim));
  double* tp = ctx->energy_scratch.p;
  double* ip = tp + ntiles;
  double* op = ip + ninst;
  energy_cells_kernel<<<ntiles, 256, 0, ctx->stream>>>(ctx->sims_d, ctx->tiles_d, ctx->cur, ctx->dt,
                                                       ctx->dx, ctx->dy, tp);
  if (ninst > 0)
    energy_rom_kernel<<<ninst, 256, 0, ctx->stream>>>(ctx->sims_d, ctx->insts_d, ctx->einst_d, ctx->cur,
                                                      ctx->dt, ip);
  energy_sum_kernel<<<nsim, 256, 0, ctx->stream>>>(tp, ctx->tile_base_d, ip, ctx->insts_d, ninst, op);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, op, sizeof(double) * nsim, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < nsim; ++k)
    if (!std::isfinite(out[k])) return fail(ctx, FDTD_EUNSTABLE, "non-finite storage function");
  return FDTD_OK;
}

int fdtd_energy_noalloc(fdtd_ctx* ctx, double* out) {
  NvtxRange nvtx_("fdtd_energy_noalloc");
  if (!ctx || !out) return fail(ctx, FDTD_EINVAL, "fdtd_energy_noalloc: bad argument");
  const int ntiles = (int)ctx->tiles.size(), ninst = (int)ctx->insts.size();
  const int nsim = (int)ctx->sims.size();
  const long long need = (long long)ntiles + ninst + nsim;
  if (need > FDTD_ENERGY_STATIC_MAX)
    return fail(ctx, FDTD_EINVAL, "fdtd_energy_noalloc: context needs " + std::to_string(need) +
                                      " partial sums, above the static capacity of " +
                                      std::to_string(FDTD_ENERGY_STATIC_MAX) + " (use fdtd_energy)");
  double* tp = nullptr;
  const int rc = static_energy_scratch(ctx, &tp);
  if (rc) return rc;
  double* ip = tp + ntiles;
  double* op = ip + ninst;
  energy_cells_kernel<<<ntiles, 256, 0, ctx->stream>>>(ctx->sims_d, ctx->tiles_d, ctx->cur, ctx->dt,
                                                       ctx->dx, ctx->dy, tp);
  if (ninst > 0)
    energy_rom_kernel<<<ninst, 256, 0, ctx->stream>>>(ctx->sims_d, ctx->insts_d, ctx->einst_d, ctx->cur,
                                                      ctx->dt, ip);
  energy_sum_kernel<<<nsim, 256, 0, ctx->stream>>>(tp, ctx->tile_base_d, ip, ctx->insts_d, ninst, op);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, op, sizeof(double) * nsim, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < nsim; ++k)
    if (!std::isfinite(out[k])) return fail(ctx, FDTD_EUNSTABLE, "non-finite storage function");
  return FDTD_OK;
}

int fdtd_grad(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc,
              const fdtd_probe* probes, int nprobe, int ckpt_every, float* dJ_deps,
              float* dJ_dsigma, float* dJ_dsrc, double* J_out) {
  NvtxRange nvtx_("fdtd_grad");
  if (!ctx) return fail(ctx, FDTD_EINVAL, "fdtd_grad: null context");
  if (ctx->timing) return fail(ctx, FDTD_EINVAL, "fdtd_grad: switch timing off first");
  return run_grad(ctx, nsteps, src, nsrc, probes, nprobe, ckpt_every, dJ_deps, dJ_dsigma, dJ_dsrc, J_out,
                  false, nullptr, nullptr);
}

int fdtd_vjp(fdtd_ctx* ctx, long long nsteps, const fdtd_source* src, int nsrc, const fdtd_probe* probes,
             int nprobe, int ckpt_every, const float* dL_dprobe, float* dL_deps, float* dL_dsigma,
             float* dL_dsrc, float* probe_out) {
  NvtxRange nvtx_("fdtd_vjp");
  if (!ctx) return fail(ctx, FDTD_EINVAL, "fdtd_vjp: null context");
  if (ctx->timing) return fail(ctx, FDTD_EINVAL, "fdtd_vjp: switch timing off first");
  if (nprobe > 0 && !dL_dprobe) return fail(ctx, FDTD_EINVAL, "fdtd_vjp: null cotangent");
  return run_grad(ctx, nsteps, src, nsrc, probes, nprobe, ckpt_every, dL_deps, dL_dsigma, dL_dsrc, nullptr,
                  true, dL_dprobe, probe_out);
}

int fdtd_autotune(fdtd_ctx* ctx, const char* cache_path, fdtd_tune_report* report) {
  NvtxRange nvtx_("fdtd_autotune");
  if (!ctx) return set_global_error(FDTD_EINVAL, "fdtd_autotune: null context");
  if (ctx->timing) return fail(ctx, FDTD_EINVAL, "fdtd_autotune: switch timing off first");
  return run_autotune(ctx, cache_path, report);
}

int fdtd_get_plan(const fdtd_ctx* ctx, fdtd_tune_report* report) {
  if (!ctx || !report) return set_global_error(FDTD_EINVAL, "fdtd_get_plan: bad argument");
  *report = fdtd_tune_report{};
  fill_report(ctx, report);
  return FDTD_OK;
}

int fdtd_set_timing(fdtd_ctx* ctx, int on) {
  if (!ctx) return set_global_error(FDTD_EINVAL, "fdtd_set_timing: null context");
  if (ctx->timing) {
    int rc = drain_events(ctx);
    if (rc) return rc;
  }
  ctx->timing = on != 0;
  ctx->t_yee = ctx->t_post = 0;
  ctx->n_yee = ctx->n_post = 0;
  ctx->ev_used = 0;
  return FDTD_OK;
}

int fdtd_steps_per_launch(const fdtd_ctx* ctx) {
  if (!ctx) return set_global_error(FDTD_EINVAL, "fdtd_steps_per_launch: null context");
  return ctx->tb ? 2 : 1;
}

int fdtd_get_kernel_times(fdtd_ctx* ctx, double* yee_ms, long long* yee_launches, double* post_ms,
                          long long* post_launches) {
  if (!ctx) return set_global_error(FDTD_EINVAL, "fdtd_get_kernel_times: null context");
  int rc = drain_events(ctx);
  if (rc) return rc;
  if (yee_ms) *yee_ms = ctx->t_yee;
  if (yee_launches) *yee_launches = ctx->n_yee;
  if (post_ms) *post_ms = ctx->t_post;
  if (post_launches) *post_launches = ctx->n_post;
  return FDTD_OK;
}

// Device time of the stencil kernel alone: a graph of back-to-back launches
// (no per-kernel events, no programmatic overlap between them) that read the
// current fields and write the other ping-pong copy, replayed reps times
// between two events.  The current fields and the step counter are not
// changed; the other copy is scratch until the next step overwrites it.
int fdtd_time_stencil(fdtd_ctx* ctx, int launches, int reps, double* ms_per_launch) {
  NvtxRange nvtx_("fdtd_time_stencil");
  if (!ctx || launches < 1 || reps < 1 || !ms_per_launch)
    return fail(ctx, FDTD_EINVAL, "fdtd_time_stencil: bad argument");
  if (ctx->timing) return fail(ctx, FDTD_EINVAL, "fdtd_time_stencil: switch timing off first");
  // run tables without sources or probes (all the stencil reads of a run)
  int rc = prepare_run(ctx, 2, nullptr, 0, nullptr, nullptr, 0, nullptr);
  if (rc) return rc;
  const int par = ctx->cur;
  const int nord = (int)ctx->tb_tiles.size() - (int)ctx->insts.size();   // shared-memory two-step: ordinary tiles
  struct Res {
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Res() {
      if (ge) cudaGraphExecDestroy(ge);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } r;
  cudaStream_t cs = ctx->capture_stream;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < launches; ++k) {
    if (ctx->tb && ctx->tb_march)
      launch_k(march_fn(ctx->tbm_mb, ctx->tbm_ring, ctx->tbm_sparse), (unsigned)ctx->tbm_tiles.size(), 32 * ctx->tbm_w,
               march_smem(ctx->tbm_ring, ctx->tbm_w), cs, false, (const SimDev*)ctx->sims_d, (const TileWork*)ctx->tbm_tiles_d, (const RunDev*)ctx->run_d,
               (const TbMarchDev*)ctx->tbm_d, par, 0, ctx->tbm_pf);
    else if (ctx->tb && nord > 0)
      yee_tb2_kernel<<<nord, kTbThreads, kTbSmemFields, cs>>>(ctx->sims_d, ctx->tb_tiles_d, ctx->insts_d, ctx->run_d,
                                                              ctx->tb_run_d, par, 0);
    else if (ctx->stencil_tma)
      yee_step_tma_kernel<<<(unsigned)ctx->tiles.size(), kCtaCols / 4, kTmaSmem, cs>>>(ctx->sims_d, ctx->tiles_d,
                                                                                      ctx->run_d, par, 0);
    else if (ctx->vec == 2)
      launch_k(yee_step_kernel<2>, (unsigned)ctx->tiles.size(), kCtaCols / 2, 0, cs, false, (const SimDev*)ctx->sims_d,
               (const TileWork*)ctx->tiles_d, (const RunDev*)ctx->run_d, par, 0);
    else
      launch_k(yee_step_kernel<4>, (unsigned)ctx->tiles.size(), kCtaCols / 4, 0, cs, false, (const SimDev*)ctx->sims_d,
               (const TileWork*)ctx->tiles_d, (const RunDev*)ctx->run_d, par, 0);
  }
  CK(cudaStreamEndCapture(cs, &g));
  const cudaError_t ei = cudaGraphInstantiate(&r.ge, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return fail(ctx, FDTD_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  CK(cudaEventCreate(&r.e0));
  CK(cudaEventCreate(&r.e1));
  CK(cudaGraphLaunch(r.ge, ctx->stream));   // warm-up replay
  CK(cudaEventRecord(r.e0, ctx->stream));
  for (int k = 0; k < reps; ++k) CK(cudaGraphLaunch(r.ge, ctx->stream));
  CK(cudaEventRecord(r.e1, ctx->stream));
  CK(cudaEventSynchronize(r.e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
  *ms_per_launch = (double)ms / ((double)reps * launches);
  return check_status(ctx);
}

// State buffer: magic, step, cur-independent field copies (Ex, Ey, Hz per
// simulation, pitched as on the device), every instance's [y; x~].
static size_t pml_psi_count(const fdtd_ctx* ctx) {
  return ctx->pml_cells.empty() ? 0 : 2 * ctx->pml_cells.size() + ctx->pml_edges.size();
}

static size_t state_bytes(const fdtd_ctx* ctx) {
  size_t b = 4 * sizeof(long long);
  for (const SimHost& sh : ctx->sims) b += 3 * sizeof(float) * (size_t)(sh.ny + 1) * sh.pitch;
  for (const Instance& in : ctx->insts) b += sizeof(float) * (size_t)in.n;
  return b + sizeof(float) * pml_psi_count(ctx);
}

int fdtd_save_state(fdtd_ctx* ctx, void* buf, size_t* size) {
  if (!ctx || !size) return fail(ctx, FDTD_EINVAL, "fdtd_save_state: bad argument");
  const size_t need = state_bytes(ctx);
  if (!buf) {
    *size = need;
    return FDTD_OK;
  }
  if (*size < need) return fail(ctx, FDTD_EINVAL, "fdtd_save_state: buffer too small");
  CK(cudaStreamSynchronize(ctx->stream));
  char* p = static_cast<char*>(buf);
  const long long hdr[4] = {0x46445444524f4d31LL, ctx->step, (long long)ctx->sims.size(), (long long)ctx->insts.size()};
  std::memcpy(p, hdr, sizeof(hdr));
  p += sizeof(hdr);
  const int c = ctx->cur;
  for (const SimHost& sh : ctx->sims) {
    const size_t bytes = sizeof(float) * (size_t)(sh.ny + 1) * sh.pitch;
    for (float* a : {sh.ex[c], sh.ey[c], sh.hz[c]}) {
      CK(cudaMemcpy(p, a, bytes, cudaMemcpyDeviceToHost));
      p += bytes;
    }
  }
  for (const Instance& in : ctx->insts) {
    CK(cudaMemcpy(p, in.state_d[c], sizeof(float) * in.n, cudaMemcpyDeviceToHost));
    p += sizeof(float) * in.n;
  }
  if (pml_psi_count(ctx)) CK(cudaMemcpy(p, ctx->pml_psi.p, sizeof(float) * pml_psi_count(ctx), cudaMemcpyDeviceToHost));
  *size = need;
  return FDTD_OK;
}

int fdtd_load_state(fdtd_ctx* ctx, const void* buf, size_t size) {
  if (!ctx || !buf) return fail(ctx, FDTD_EINVAL, "fdtd_load_state: bad argument");
  const size_t need = state_bytes(ctx);
  long long hdr[4];
  if (size != need) return fail(ctx, FDTD_EINVAL, "fdtd_load_state: size does not match this context");
  std::memcpy(hdr, buf, sizeof(hdr));
  if (hdr[0] != 0x46445444524f4d31LL || hdr[2] != (long long)ctx->sims.size() ||
      hdr[3] != (long long)ctx->insts.size())
    return fail(ctx, FDTD_EINVAL, "fdtd_load_state: buffer was saved from another layout");
  CK(cudaStreamSynchronize(ctx->stream));
  const char* p = static_cast<const char*>(buf) + sizeof(hdr);
  const int c = ctx->cur;
  for (const SimHost& sh : ctx->sims) {
    const size_t bytes = sizeof(float) * (size_t)(sh.ny + 1) * sh.pitch;
    for (float* a : {sh.ex[c], sh.ey[c], sh.hz[c]}) {
      CK(cudaMemcpy(a, p, bytes, cudaMemcpyHostToDevice));
      p += bytes;
    }
  }
  for (const Instance& in : ctx->insts) {
    CK(cudaMemcpy(in.state_d[c], p, sizeof(float) * in.n, cudaMemcpyHostToDevice));
    p += sizeof(float) * in.n;
  }
  if (pml_psi_count(ctx)) CK(cudaMemcpy(ctx->pml_psi.p, p, sizeof(float) * pml_psi_count(ctx), cudaMemcpyHostToDevice));
  ctx->step = hdr[1];
  return FDTD_OK;
}

int fdtd_selftest_timeout(fdtd_ctx* ctx) {
  if (!ctx) return set_global_error(FDTD_EINVAL, "fdtd_selftest_timeout: null context");
  CK(cudaStreamSynchronize(ctx->stream));
  int rc = check_status(ctx);   // report anything earlier first
  if (rc) return rc;
  wait_selftest_kernel<<<1, 64, 0, ctx->stream>>>(ctx->status_d, 1000u);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

int fdtd_set_pml(fdtd_ctx* ctx, int sim, const fdtd_pml_desc* pd) {
  if (!ctx || !pd || sim < 0 || sim >= (int)ctx->sims.size())
    return fail(ctx, FDTD_EINVAL, "fdtd_set_pml: bad argument");
  const SimHost& sh = ctx->sims[sim];
  fdtd_pml_desc d = *pd;
  if (d.sides < 0 || d.sides > 15) return fail(ctx, FDTD_EINVAL, "fdtd_set_pml: bad sides");
  if (d.sides != 0) {
    const int n = d.ncells;
    const int lx = ((d.sides & FDTD_PML_W) ? n : 0) + ((d.sides & FDTD_PML_E) ? n : 0);
    const int ly = ((d.sides & FDTD_PML_S) ? n : 0) + ((d.sides & FDTD_PML_N) ? n : 0);
    if (n < 1 || lx > sh.nx - 2 || ly > sh.ny - 2)
      return fail(ctx, FDTD_EINVAL, "fdtd_set_pml: layers must leave two interior cells");
    if (!(d.m > 0) || !(d.kappa_max >= 1) || !(d.alpha_max >= 0) || !std::isfinite(d.sigma_max))
      return fail(ctx, FDTD_EINVAL, "fdtd_set_pml: bad profile");
  }
  if ((int)ctx->pml_desc.size() < (int)ctx->sims.size()) {
    fdtd_pml_desc none{};
    ctx->pml_desc.resize(ctx->sims.size(), none);
    ctx->pml_coef.resize(ctx->sims.size());
  }
  const fdtd_pml_desc old = ctx->pml_desc[sim];
  ctx->pml_desc[sim] = d;
  for (const Instance& in : ctx->insts) {
    if (in.sim != sim) continue;
    for (int j = in.j0 - 2; j < in.j0 + in.b + 2; ++j)
      for (int i = in.i0 - 2; i < in.i0 + in.a + 2; ++i)
        if (pml_cell(ctx, sim, i, j)) {
          ctx->pml_desc[sim] = old;
          return fail(ctx, FDTD_EINVAL, "fdtd_set_pml: a layer comes within two cells of an embedded region");
        }
  }
  // coefficient arrays of this simulation, FP64 then rounded
  std::vector<float>& cf = ctx->pml_coef[sim];
  cf.clear();
  if (d.sides != 0) {
    const double eta0 = std::sqrt(kMu0 / kEps0), dt = ctx->dt;
    auto arr = [&](int len, double off, int extent, bool lo, bool hi, double h) {
      const double smax = d.sigma_max > 0 ? d.sigma_max : 0.8 * (d.m + 1) / (eta0 * h);
      std::vector<float> b(len), a(len), rk(len);
      for (int k = 0; k < len; ++k) {
        const double pos = k + off;
        double dep = 0;
        if (lo) dep = std::max(dep, d.ncells - pos);
        if (hi) dep = std::max(dep, pos - (extent - d.ncells));
        const double rho = std::min(std::max(dep, 0.0), (double)d.ncells) / d.ncells;
        double sg = 0, kp = 1, al = 0;
        if (rho > 0) {
          sg = smax * std::pow(rho, d.m);
          kp = 1 + (d.kappa_max - 1) * std::pow(rho, d.m);
          al = d.alpha_max * (1 - rho);
        }
        const double bb = std::exp(-(sg / kp + al) * dt / kEps0);
        const double den = sg * kp + kp * kp * al;
        b[k] = (float)bb;
        a[k] = (float)(sg > 0 ? sg / den * (bb - 1) : 0.0);
        rk[k] = (float)(1.0 / kp);
      }
      cf.insert(cf.end(), b.begin(), b.end());
      cf.insert(cf.end(), a.begin(), a.end());
      cf.insert(cf.end(), rk.begin(), rk.end());
    };
    const bool W = d.sides & FDTD_PML_W, E = d.sides & FDTD_PML_E, S = d.sides & FDTD_PML_S,
               N = d.sides & FDTD_PML_N;
    arr(sh.nx, 0.5, sh.nx, W, E, ctx->dx);       // xh: Hz, Ex columns at (i + 1/2) dx
    arr(sh.ny, 0.5, sh.ny, S, N, ctx->dy);       // yh: Hz, Ey rows at (j + 1/2) dy
    arr(sh.nx + 1, 0.0, sh.nx, W, E, ctx->dx);   // xe: Ey columns at i dx
    arr(sh.ny + 1, 0.0, sh.ny, S, N, ctx->dy);   // ye: Ex rows at j dy
  }
  // lists and device tables of every simulation
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->pml_cells.clear();
  std::vector<int2> exl, eyl;
  std::vector<PmlSimDev> tab(ctx->sims.size());
  std::vector<float> coef;
  std::vector<size_t> coff(ctx->sims.size(), 0);
  for (int t = 0; t < (int)ctx->sims.size(); ++t) {
    coff[t] = coef.size();
    coef.insert(coef.end(), ctx->pml_coef[t].begin(), ctx->pml_coef[t].end());
    const fdtd_pml_desc& dt_ = ctx->pml_desc[t];
    if (dt_.sides == 0) continue;
    const SimHost& st = ctx->sims[t];
    for (int j = 0; j < st.ny; ++j)
      for (int i = 0; i < st.nx; ++i)
        if (pml_cell(ctx, t, i, j)) ctx->pml_cells.push_back(make_int2(t, j * st.pitch + i));
    for (int j = 1; j < st.ny; ++j)
      for (int i = 0; i < st.nx; ++i)
        if (edge_updated(st, 0, i, j) && pml_edge(ctx, t, 0, i, j)) exl.push_back(make_int2(t, j * st.pitch + i));
    for (int j = 0; j < st.ny; ++j)
      for (int i = 1; i < st.nx; ++i)
        if (edge_updated(st, 1, i, j) && pml_edge(ctx, t, 1, i, j)) eyl.push_back(make_int2(t, j * st.pitch + i));
  }
  ctx->pml_nex = (int)exl.size();
  ctx->pml_edges = exl;
  ctx->pml_edges.insert(ctx->pml_edges.end(), eyl.begin(), eyl.end());
  const size_t nc = ctx->pml_cells.size(), ne = ctx->pml_edges.size();
  if (nc > 0) {
    CK(ctx->pml_coef_d.reserve(coef.size()));
    CK(cudaMemcpy(ctx->pml_coef_d.p, coef.data(), sizeof(float) * coef.size(), cudaMemcpyHostToDevice));
    for (int t = 0; t < (int)ctx->sims.size(); ++t) {
      const SimHost& st = ctx->sims[t];
      PmlSimDev& pm = tab[t];
      pm = PmlSimDev{};
      if (ctx->pml_coef[t].empty()) continue;
      const float* base = ctx->pml_coef_d.p + coff[t];
      pm.nxh = st.nx, pm.nyh = st.ny, pm.nxe = st.nx + 1, pm.nye = st.ny + 1;
      pm.xh = base;
      pm.yh = pm.xh + 3 * pm.nxh;
      pm.xe = pm.yh + 3 * pm.nyh;
      pm.ye = pm.xe + 3 * pm.nxe;
      pm.dtmu = (float)(ctx->dt / kMu0);
    }
    CK(ctx->pml_sims_d.reserve(tab.size()));
    CK(cudaMemcpy(ctx->pml_sims_d.p, tab.data(), sizeof(PmlSimDev) * tab.size(), cudaMemcpyHostToDevice));
    CK(ctx->pml_cells_d.reserve(nc));
    CK(cudaMemcpy(ctx->pml_cells_d.p, ctx->pml_cells.data(), sizeof(int2) * nc, cudaMemcpyHostToDevice));
    CK(ctx->pml_edges_d.reserve(std::max<size_t>(ne, 1)));
    if (ne) CK(cudaMemcpy(ctx->pml_edges_d.p, ctx->pml_edges.data(), sizeof(int2) * ne, cudaMemcpyHostToDevice));
    CK(ctx->pml_psi.reserve(2 * nc + ne));
    CK(cudaMemset(ctx->pml_psi.p, 0, sizeof(float) * (2 * nc + ne)));
  }
  drop_graphs(ctx);
  return plan_tb(ctx);
}

int fdtd_fine_fields(fdtd_ctx* ctx, int inst, const rom_model* m, float* Ex, float* Ey, float* Hz) {
  if (!ctx || !m || !Ex || !Ey || !Hz || inst < 0 || inst >= (int)ctx->insts.size())
    return fail(ctx, FDTD_EINVAL, "fdtd_fine_fields: bad argument");
  const Instance& in = ctx->insts[inst];
  if (in.map->model_id != m->id)
    return fail(ctx, FDTD_EINVAL, "fdtd_fine_fields: instance was embedded with another model");
  const int nE = m->V1.r, nH = m->V2.r, qE = m->V1.c, qH = m->V2.c;
  const int nEx = m->nxf * (m->nyf + 1);
  fdtd_ctx::Basis* b = nullptr;
  for (auto& x : ctx->bases)
    if (x.id == m->id) b = &x;
  if (!b) {
    fdtd_ctx::Basis nb{m->id, nullptr, nullptr};
    std::vector<float> h1(m->V1.a.begin(), m->V1.a.end()), h2(m->V2.a.begin(), m->V2.a.end());
    CK(cudaMalloc(&nb.V1, sizeof(float) * std::max<size_t>(h1.size(), 1)));
    if (cudaMalloc(&nb.V2, sizeof(float) * std::max<size_t>(h2.size(), 1)) != cudaSuccess) {
      cudaFree(nb.V1);
      return fail(ctx, FDTD_ENOMEM, "fdtd_fine_fields: device allocation failed");
    }
    ctx->bases.push_back(nb);
    b = &ctx->bases.back();
    CK(cudaMemcpy(b->V1, h1.data(), sizeof(float) * h1.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->V2, h2.data(), sizeof(float) * h2.size(), cudaMemcpyHostToDevice));
  }
  const float* xt = in.state_d[ctx->cur] + in.ny;   // x~ follows y in [y; x~]
  const int rows = nE + nH;
  const unsigned nb = (unsigned)std::min(1024, (rows + 7) / 8);
  fine_fields_kernel<<<nb, 256, sizeof(float) * std::max(qE + qH, 1), ctx->stream>>>(
      b->V1, b->V2, xt, nE, nH, qE, qH, nEx, Ex, Ey, Hz);
  CK(cudaGetLastError());
  return FDTD_OK;
}

int fdtd_dft_set(fdtd_ctx* ctx, const fdtd_probe* mons, int nmon, const double* freqs, int nfreq,
                 const double* acc_init) {
  if (!ctx || nmon < 0 || nfreq < 0 || (nmon > 0 && (!mons || !freqs || nfreq < 1)))
    return fail(ctx, FDTD_EINVAL, "fdtd_dft_set: bad argument");
  if ((long long)nmon * nfreq > (1ll << 24))
    return fail(ctx, FDTD_EINVAL, "fdtd_dft_set: more than 2^24 monitor-frequency pairs");
  std::vector<int> sim(nmon), cell(nmon);
  for (int m = 0; m < nmon; ++m) {
    if (mons[m].sim < 0 || mons[m].sim >= (int)ctx->sims.size())
      return fail(ctx, FDTD_EINVAL, "fdtd_dft_set: monitor sim out of range");
    const SimHost& sh = ctx->sims[mons[m].sim];
    if (mons[m].i < 0 || mons[m].i >= sh.nx || mons[m].j < 0 || mons[m].j >= sh.ny)
      return fail(ctx, FDTD_EINVAL, "fdtd_dft_set: monitor outside the grid");
    sim[m] = mons[m].sim;
    cell[m] = mons[m].j * sh.pitch + mons[m].i;
  }
  std::vector<double> fdt(nfreq);
  for (int f = 0; f < nfreq && nmon > 0; ++f) {
    if (!std::isfinite(freqs[f]) || freqs[f] < 0)
      return fail(ctx, FDTD_EINVAL, "fdtd_dft_set: frequencies must be finite and >= 0");
    fdt[f] = freqs[f] * ctx->dt;
  }
  CK(cudaStreamSynchronize(ctx->stream));   // no run may be using the old tables
  ctx->dft_nmon = 0;
  ctx->dft_nfreq = 0;
  if (nmon == 0) return FDTD_OK;
  const size_t np = (size_t)nmon * nfreq;
  CK(ctx->dft_sim.reserve(nmon));
  CK(ctx->dft_cell.reserve(nmon));
  CK(ctx->dft_fdt.reserve(nfreq));
  CK(ctx->dft_acc.reserve(np));
  CK(cudaMemcpy(ctx->dft_sim.p, sim.data(), sizeof(int) * nmon, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->dft_cell.p, cell.data(), sizeof(int) * nmon, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->dft_fdt.p, fdt.data(), sizeof(double) * nfreq, cudaMemcpyHostToDevice));
  std::vector<double2> acc(np, make_double2(0.0, 0.0));
  if (acc_init)
    for (size_t k = 0; k < np; ++k) acc[k] = make_double2(acc_init[2 * k] / ctx->dt, acc_init[2 * k + 1] / ctx->dt);
  CK(cudaMemcpy(ctx->dft_acc.p, acc.data(), sizeof(double2) * np, cudaMemcpyHostToDevice));
  ctx->dft_nmon = nmon;
  ctx->dft_nfreq = nfreq;
  return FDTD_OK;
}

int fdtd_dft_get(fdtd_ctx* ctx, double* out) {
  if (!ctx || (!out && ctx->dft_nmon > 0)) return fail(ctx, FDTD_EINVAL, "fdtd_dft_get: bad argument");
  const size_t np = (size_t)ctx->dft_nmon * ctx->dft_nfreq;
  if (np == 0) return FDTD_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(out, ctx->dft_acc.p, sizeof(double2) * np, cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < 2 * np; ++k) out[k] *= ctx->dt;
  return FDTD_OK;
}

int fdtd_get_step(const fdtd_ctx* ctx, long long* n) {
  if (!ctx || !n) return set_global_error(FDTD_EINVAL, "fdtd_get_step: bad argument");
  *n = ctx->step;
  return FDTD_OK;
}

}  // extern "C"
