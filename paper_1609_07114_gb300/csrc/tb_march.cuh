// Two time steps per pass without shared memory (temporal blocking by row
// marching).  Included by fdtd.cu after tb.cuh.
//
// A warp owns kMarchOut = 120 output columns [c0, c0 + 120) of a tile and
// computes the 128 columns [c0 - 4, c0 + 124): lane l holds columns
// c0 - 4 + 4 l .. + 3, so the left two and right one halo columns that two
// steps need are ordinary lane columns (lanes 0 and 31) and every neighbour
// value comes from a shuffle; values in the outermost columns of lanes 0 and
// 31 are wrong (their shuffles wrap) but nothing stored depends on them.  A
// CTA has W = 3 or 4 warps (blockDim.x / 32, the plan's choice: the fewer
// idle warps in the grids' last column blocks) and a tile W x 120 columns.
// Marching up the rows, iteration j computes
//   A: row j of Hz^{n+1/2}, Ex^{n+1}, Ey^{n+1} from E^n, Hz^{n-1/2} (Eq. (5),
//      then Eq. (3), sources J^n), and
//   B: row j - 1 of Hz^{n+3/2}, Ex^{n+2}, Ey^{n+2} from rows j - 1, j of A
//      (sources J^{n+1}); the edge coefficients of row j - 1 are those A
//      computed one row earlier,
// holding everything in registers, and stores B's row when the tile owns it.
// A starts two rows below the tile and B one row below, so the tile's first
// stored row has all it needs.  Each update is the same sequence of explicit
// operations as stencil_row (correctly rounded products and sums, the
// hardware reciprocal of edge_coef), so two passes of this kernel give the
// bits of four launches of the one-step kernel.
//
// Model regions: the cells of each model's zone (the region grown by three
// cells, columns rounded out to multiples of 4) are stepped by the in-CTA
// model tiles of yee_tb2_kernel, which evaluate the coupling between the
// sub-steps; this kernel computes through zones without the coupling but
// does not store zone cells (over two steps an error at the interface reaches
// at most two cells).  Probes in zones are written by the model tiles too.

namespace {

constexpr int kMarchOut = 120;                // output columns per warp

struct MarchSrc {   // a driven edge within a warp's computed columns and rows
  int j, i;
  int cs;           // comp | src << 1 (a warp's entries: rows ascending, Ex before Ey)
  float cb;         // the edge's cb (march_src_cb_kernel, the stencil's own operations)
};
constexpr int kMarchNone = 0x7fffffff;   // row of the end-of-list entry

struct MarchPrb {   // a probe cell owned by a warp (outside every zone)
  int j, i, p, pad;
};

struct TbMarchDev {
  const int2* src_rng;    // per warp (tile * W + warp): [begin, end) into src, rows ascending
  const MarchSrc* src;
  const int2* prb_rng;    // per warp: [begin, end) into prb, rows ascending
  const MarchPrb* prb;
  const int2* zone_rng;   // per tile: [begin, end) into zones
  const int4* zones;      // x0, y0, x1, y1 (x0 a multiple of 4)
};

struct MarchIn {        // the loads of row j for sub-step A
  float4 exn, eyv, hzv; // Ex^n(j + 1), Ey^n(j), Hz^{n-1/2}(j)
  float4 ma, mb;        // mat(j) of the lane's 4 cells
};

// Sparse materials: whether row j of the warp's 128 columns [c0 - 4, c0 + 124),
// which lie in at most two of the 128-column strips of the simulation's bits,
// holds a cell other than the background (or the cell left of a strip does).
// The warp gathers the words of its tile's rows (one per 32 rows, both strips
// OR-ed) into shared memory once; a row's bit is then one shared load.
// Warp-uniform.
constexpr int kMarchBitWords = 4096 / 32 + 3;   // tiles of up to 4096 rows (FDTD_TB_ROWS is clamped to that)

__device__ __forceinline__ void march_gather_bits(uint32_t* sbits, const SimDev& sd, int jA0, int jAe, int c0,
                                                  int lane) {
  const int jw0 = jA0 >> 5;
  const int nw = min((jAe >> 5) - jw0 + 1, kMarchBitWords);
  const int s0 = max(c0 - 4, 0) >> 7, s1 = min(c0 + 123, sd.pitch - 1) >> 7;
  for (int k = lane; k < nw; k += 32) {
    const int wj = jw0 + k;
    uint32_t b = 0xffffffffu;   // rows past the grid are not loaded anyway
    if (wj <= ((sd.ny - 1) >> 5)) {
      const uint32_t* w = sd.mbits + (size_t)wj * sd.nstrip;
      b = w[s0] | w[s1];
    }
    sbits[k] = b;
  }
  __syncwarp();
}

__device__ __forceinline__ bool march_dense(const uint32_t* sbits, int j, int jw0) {
  return ((sbits[(j >> 5) - jw0] >> (j & 31)) & 1u) != 0u;
}

// Lanes outside the pitched row and rows >= ny read nothing (dead cells);
// rows of background cells only (dense false) take the background material
// without reading it.
__device__ __forceinline__ void march_load(MarchIn& r, const float* __restrict__ ex,
                                           const float* __restrict__ ey, const float* __restrict__ hz,
                                           const float2* __restrict__ mat, int j, int ny, int P, int cl,
                                           bool inb, bool dense, const float2* __restrict__ bgp) {
  if (inb && j < ny) {
    const size_t row = (size_t)j * P + cl;
    r.exn = ld4(ex + row + P);
    r.eyv = ld4(ey + row);
    r.hzv = ld4(hz + row);
    if (dense) {
      r.ma = ld4(reinterpret_cast<const float*>(mat + row));
      r.mb = ld4(reinterpret_cast<const float*>(mat + row + 2));
    } else {
      const float2 bg = *bgp;
      r.ma = r.mb = make_float4(bg.x, bg.y, bg.x, bg.y);
    }
  } else {
    r.exn = r.eyv = r.hzv = make_float4(0.f, 0.f, 0.f, 0.f);
    r.ma = r.mb = make_float4(-1.f, 0.f, -1.f, 0.f);
  }
}

// E -= cb J on the edge of column i if the lane holds it.
__device__ __forceinline__ void march_source(float (&e)[4], const MarchSrc& s, int cl, float J) {
  const int t = s.i - cl;
  const float d = __fmul_rn(s.cb, J);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q == t) e[q] = __fsub_rn(e[q], d);
}

// The next list entry (loaded one row before it is needed).
__device__ __forceinline__ MarchSrc march_src_at(const MarchSrc* __restrict__ src, int k, int e) {
  if (k < e) return src[k];
  MarchSrc n;
  n.j = kMarchNone, n.i = 0, n.cs = 0, n.cb = 0.f;
  return n;
}
__device__ __forceinline__ MarchPrb march_prb_at(const MarchPrb* __restrict__ prb, int k, int e) {
  if (k < e) return prb[k];
  MarchPrb n;
  n.j = kMarchNone, n.i = 0, n.p = 0, n.pad = 0;
  return n;
}

// cb of every list entry from the two cells beside its edge (edge_coef, as
// the stencil forms it), once per run.
__global__ void march_src_cb_kernel(const SimDev* __restrict__ sims, const int* __restrict__ ent_sim,
                                    MarchSrc* __restrict__ src, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const SimDev sd = sims[ent_sim[k]];
  MarchSrc s = src[k];
  const size_t off = (size_t)s.j * sd.pitch + s.i;
  float ca, cb;
  edge_coef((s.cs & 1) == 0 ? sd.mat[off - sd.pitch] : sd.mat[off - 1], sd.mat[off], ca, cb);
  src[k].cb = cb;
}

// L2 prefetch of the loads of row j (TMA-engine bulk prefetch: 16-byte
// aligned start, size a multiple of 16, clipped to the pitched row).
__device__ __forceinline__ void march_prefetch(const float* ex, const float* ey, const float* hz,
                                               const float2* mat, int j, int P, int c0, int lane) {
  const int n = min(128, P - c0) & ~3;
  const size_t row = (size_t)j * P + c0;
  const void* p = nullptr;
  unsigned bytes = 4u * n;
  if (lane == 0) p = ex + row + P;
  else if (lane == 1) p = ey + row;
  else if (lane == 2) p = hz + row;
  else if (lane == 3) p = mat + row, bytes = 8u * n;
  if (p && bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L1 prefetch of the lane's part of row j (each lane its own 16-byte pieces;
// no registers held).
__device__ __forceinline__ void march_prefetch_l1(const float* ex, const float* ey, const float* hz,
                                                  const float2* mat, int j, int P, int cl) {
  const size_t row = (size_t)j * P + cl;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(ex + row + P));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(ey + row));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(hz + row));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(mat + row));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(mat + row + 2));
}

__device__ __forceinline__ float pick4(const float (&v)[4], int t) {
  return t == 0 ? v[0] : (t == 1 ? v[1] : (t == 2 ? v[2] : v[3]));
}

// Staged form of the loads (kRing >= 2 rows): each lane copies its own five
// float4 of a row into its warp's ring in shared memory with cp.async, kRing - 1
// rows ahead of the row it computes, one commit group per row; the copies in
// flight hold no registers and the compiler cannot sink them.  A lane reads
// back only what it copied itself, so waiting on its own groups suffices.
// Ring layout: [warp][slot][5 values][32 lanes] float4.
constexpr int kMarchRingBytesPerRow = 4 * 5 * 32 * 16;   // four warps

__device__ __forceinline__ void march_issue(float4* slot, const float* __restrict__ ex, const float* __restrict__ ey,
                                            const float* __restrict__ hz, const float2* __restrict__ mat, int j, int ny,
                                            int P, int cl, bool inb, int lane, bool dense) {
  asm volatile("" ::: "memory");   // after the reads of the slot's previous row
  const bool ok = inb && j < ny;
  const size_t row = ok ? (size_t)j * P + cl : 0;
  cp_async16(slot + 0 * 32 + lane, ok ? ex + row + P : ex, ok);
  cp_async16(slot + 1 * 32 + lane, ey + row, ok);
  cp_async16(slot + 2 * 32 + lane, hz + row, ok);
  if (dense) {
    cp_async16(slot + 3 * 32 + lane, mat + row, ok);
    cp_async16(slot + 4 * 32 + lane, mat + row + 2, ok);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void march_fetch(MarchIn& r, const float4* slot, int j, int ny, bool inb, int lane,
                                            bool dense, const float2* __restrict__ bgp) {
  if (inb && j < ny) {
    r.exn = slot[0 * 32 + lane];
    r.eyv = slot[1 * 32 + lane];
    r.hzv = slot[2 * 32 + lane];
    if (dense) {
      r.ma = slot[3 * 32 + lane];
      r.mb = slot[4 * 32 + lane];
    } else {
      const float2 bg = *bgp;
      r.ma = r.mb = make_float4(bg.x, bg.y, bg.x, bg.y);
    }
  } else {
    r.exn = r.eyv = r.hzv = make_float4(0.f, 0.f, 0.f, 0.f);
    r.ma = r.mb = make_float4(-1.f, 0.f, -1.f, 0.f);
  }
}

template <int N>
__device__ __forceinline__ void cp_async_wait_n() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int kMinBlocks, int kRing, bool kSparse, bool kFrames = false>
__global__ void __launch_bounds__(128, kMinBlocks)
yee_tb2m_kernel(const SimDev* __restrict__ sims, const TileWork* __restrict__ tiles,
                const RunDev* __restrict__ run, const TbMarchDev* __restrict__ tm, int par, int c, int pf) {
  extern __shared__ float4 march_ring[];
  const unsigned FULL = 0xffffffffu;
  const TileWork tw = tiles[blockIdx.x];
  const SimDev sd = sims[tw.sim];
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = tw.x0 + kMarchOut * warp;
  const int nx = sd.nx, ny = sd.ny, P = sd.pitch;
  if (c0 >= nx) return;
  const float* __restrict__ ex = par ? sd.ex[1] : sd.ex[0];
  const float* __restrict__ ey = par ? sd.ey[1] : sd.ey[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  float* __restrict__ exo = par ? sd.ex[0] : sd.ex[1];
  float* __restrict__ eyo = par ? sd.ey[0] : sd.ey[1];
  float* __restrict__ hzo = par ? sd.hz[0] : sd.hz[1];
  const float2* __restrict__ mat = sd.mat;
  const int cl = c0 - 4 + 4 * lane;
  const bool inb = cl >= 0 && cl < P;
  const bool owner = lane >= 1 && lane <= 30 && cl < nx;
  const int j0 = tw.y0, j1 = tw.y1;
  const int jA0 = j0 >= 2 ? j0 - 2 : 0, jAe = j1 < ny ? j1 : ny, jB0 = j0 >= 1 ? j0 - 1 : 0;
  const long long nA = run->base + 2 * (long long)c, nB = nA + 1;
  const int nprobe = run->nprobe;
  const int wi = blockIdx.x * (blockDim.x >> 5) + warp;
  const int2 sr = tm->src_rng[wi], pr = tm->prb_rng[wi], zr = tm->zone_rng[blockIdx.x];
  int kA = sr.x, kB = sr.x, pA = pr.x, pB = pr.x;
  while (kB < sr.y && tm->src[kB].j < jB0) ++kB;
  // next entries in registers; the samples J^n, J^{n+1} of the last source seen
  MarchSrc sa = march_src_at(tm->src, kA, sr.y), sb = march_src_at(tm->src, kB, sr.y);
  MarchPrb qa = march_prb_at(tm->prb, pA, pr.y), qb = qa;
  int jsrc = -1;
  float JA = 0.f, JB = 0.f;
  auto samples = [&](int cs) {
    if ((cs >> 1) != jsrc) {
      jsrc = cs >> 1;
      const float* __restrict__ wv = run->waves[jsrc];
      JA = wv[nA];
      JB = wv[nB];
    }
  };

  // carried state (module header): A's Ex^n(j), Hz^{n+1/2}(j-1), mat(j-1);
  // B's Ex^{n+1}(j-1), Ey^{n+1}(j-1), Hz^{n+3/2}(j-2) and the coefficients
  // (ca, cb/dy | cb/dx) of row j-1's edges with their update bits
  float exc[4], hzp[4], xaP[4], yaP[4], hbP[4], cxa[4], cxr[4], cya[4], cyr[4];
  float2 mp[4];
  unsigned lmask = 0;
  {
    const float4 e = inb ? ld4(ex + (size_t)jA0 * P + cl) : make_float4(0.f, 0.f, 0.f, 0.f);
    exc[0] = e.x, exc[1] = e.y, exc[2] = e.z, exc[3] = e.w;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      hzp[t] = xaP[t] = yaP[t] = hbP[t] = cxa[t] = cxr[t] = cya[t] = cyr[t] = 0.f;
      mp[t] = make_float2(-1.f, 0.f);
    }
  }
  MarchIn cur, nxt;
  // sparse-material bits of the row being loaded; the background material
  const float2* __restrict__ bg = &sims[tw.sim].mbg;
  __shared__ uint32_t march_bits[kSparse ? 4 : 1][kSparse ? kMarchBitWords : 1];
  uint32_t* sbits = march_bits[kSparse ? warp : 0];
  const int jw0 = jA0 >> 5;
  if constexpr (kSparse) march_gather_bits(sbits, sd, jA0, jAe, c0, lane);
  float4* ring = march_ring + (size_t)warp * (kRing > 0 ? kRing : 1) * 5 * 32;
  int slot = 0;
  unsigned dslots = 0;   // ring: slot k holds a row whose materials were read
  if constexpr (kRing > 0) {
#pragma unroll
    for (int d = 0; d < kRing - 1; ++d) {
      const bool dn = !kSparse || march_dense(sbits, jA0 + d, jw0);
      dslots = dn ? dslots | (1u << d) : dslots & ~(1u << d);
      march_issue(ring + d * 5 * 32, ex, ey, hz, mat, jA0 + d, ny, P, cl, inb, lane, dn);
    }
  } else {
    march_load(cur, ex, ey, hz, mat, jA0, ny, P, cl, inb, !kSparse || march_dense(sbits, jA0, jw0), bg);
  }
  for (int j = jA0; j <= jAe; ++j) {
    if constexpr (kRing > 0) {
      int ahead = slot + kRing - 1;
      ahead -= ahead >= kRing ? kRing : 0;
      // row j + kRing - 1 (past the tile: an empty group, so the count stays uniform)
      if (j + kRing - 1 <= jAe) {
        const bool dn = !kSparse || march_dense(sbits, j + kRing - 1, jw0);
        dslots = dn ? dslots | (1u << ahead) : dslots & ~(1u << ahead);
        march_issue(ring + ahead * 5 * 32, ex, ey, hz, mat, j + kRing - 1, ny, P, cl, inb, lane, dn);
      } else {
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
      cp_async_wait_n<kRing - 1>();
      march_fetch(cur, ring + slot * 5 * 32, j, ny, inb, lane, ((dslots >> slot) & 1u) != 0u, bg);
      slot = slot + 1 == kRing ? 0 : slot + 1;
    } else {
      if (pf > 0 && j + pf <= jAe && j + pf < ny) march_prefetch(ex, ey, hz, mat, j + pf, P, c0, lane);
      if (pf < 0 && j - pf <= jAe && j - pf < ny && inb) march_prefetch_l1(ex, ey, hz, mat, j - pf, P, cl);
      if (j + 1 <= jAe)
        march_load(nxt, ex, ey, hz, mat, j + 1, ny, P, cl, inb, !kSparse || march_dense(sbits, j + 1, jw0),
                   bg);
    }
    const float2 m[4] = {make_float2(cur.ma.x, cur.ma.y), make_float2(cur.ma.z, cur.ma.w),
                         make_float2(cur.mb.x, cur.mb.y), make_float2(cur.mb.z, cur.mb.w)};
    // ---- A.H: Hz^{n+1/2}(j) (Eq. (5))
    float eyA[5] = {cur.eyv.x, cur.eyv.y, cur.eyv.z, cur.eyv.w, 0.f};
    eyA[4] = __shfl_down_sync(FULL, eyA[0], 1);
    float hn[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const bool live = (cl + t < nx) && (m[t].x >= 0.f);
      hn[t] = live ? __fsub_rn(__fmaf_rn(sd.chx, __fsub_rn(comp(cur.exn, t), exc[t]), comp(cur.hzv, t)),
                               __fmul_rn(sd.chy, __fsub_rn(eyA[t + 1], eyA[t])))
                   : 0.f;
    }
    while (qa.j == j) {
      const int t = qa.i - cl;
      if (t >= 0 && t < 4) run->probe_out[nA * nprobe + qa.p] = pick4(hn, t);
      qa = march_prb_at(tm->prb, ++pA, pr.y);
    }
    // ---- A.Ex: Ex^{n+1}(j), edges between cells (i, j-1) and (i, j) (Eq. (3))
    // (branch-free: the coefficients are formed for every edge and the
    // update selected where the edge is updated; the carried coefficients of
    // edges that are not are never used)
    float xa[4], nxa[4], nxr[4];
    unsigned nmask = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float ca, r;
      edge_coef_r(mp[t], m[t], ca, r);
      nxa[t] = ca;
      nxr[t] = __fmul_rn(r, sd.rdy2);
      const float v = __fmaf_rn(ca, exc[t], __fmul_rn(nxr[t], __fsub_rn(hn[t], hzp[t])));
      const bool upd = j >= 1 && cl + t < nx && mp[t].x >= 0.f && m[t].x >= 0.f;
      xa[t] = upd ? v : exc[t];
      nmask |= upd ? 1u << t : 0u;
    }
    while (sa.j == j && (sa.cs & 1) == 0) {
      samples(sa.cs);
      march_source(xa, sa, cl, JA);
      sa = march_src_at(tm->src, ++kA, sr.y);
    }
    // ---- B at row r = j - 1: Hz^{n+3/2}(r), then Ex^{n+2}(r), Ey^{n+2}(r)
    const int r = j - 1;
    if (r >= jB0) {
      const float yR = __shfl_down_sync(FULL, yaP[0], 1);
      float hb[4], xb[4], yb[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const bool live = (cl + t < nx) && (mp[t].x >= 0.f);
        const float yr = t < 3 ? yaP[t + 1] : yR;
        hb[t] = live ? __fsub_rn(__fmaf_rn(sd.chx, __fsub_rn(xa[t], xaP[t]), hzp[t]),
                                 __fmul_rn(sd.chy, __fsub_rn(yr, yaP[t])))
                     : 0.f;
      }
      while (qb.j == r) {
        const int t = qb.i - cl;
        if (t >= 0 && t < 4) run->probe_out[nB * nprobe + qb.p] = pick4(hb, t);
        qb = march_prb_at(tm->prb, ++pB, pr.y);
      }
      const float hL = __shfl_up_sync(FULL, hb[3], 1);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        xb[t] = ((lmask >> t) & 1u) ? __fmaf_rn(cxa[t], xaP[t], __fmul_rn(cxr[t], __fsub_rn(hb[t], hbP[t])))
                                    : xaP[t];
        const float hl = t == 0 ? hL : hb[t - 1];
        yb[t] = ((lmask >> (4 + t)) & 1u)
                    ? __fmaf_rn(cya[t], yaP[t], -__fmul_rn(cyr[t], __fsub_rn(hb[t], hl)))
                    : yaP[t];
      }
      while (sb.j == r) {
        samples(sb.cs);
        if ((sb.cs & 1) == 0) march_source(xb, sb, cl, JB);
        else march_source(yb, sb, cl, JB);
        sb = march_src_at(tm->src, ++kB, sr.y);
      }
      bool store = owner && r >= j0;
      for (int z = zr.x; z < zr.y; ++z) {
        const int4 zn = tm->zones[z];
        if (r >= zn.y && r < zn.w && cl < zn.z && cl + 4 > zn.x) store = false;
      }
      if (store) {
        const size_t off = (size_t)r * P + cl;
        st4(hzo + off, make_float4(hb[0], hb[1], hb[2], hb[3]));
        st4(exo + off, make_float4(xb[0], xb[1], xb[2], xb[3]));
        st4(eyo + off, make_float4(yb[0], yb[1], yb[2], yb[3]));
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) hbP[t] = hb[t];
    }
    // ---- A.Ey: Ey^{n+1}(j), edges between cells (i-1, j) and (i, j)
    const float hl0 = __shfl_up_sync(FULL, hn[3], 1);
    const float2 mL = make_float2(__shfl_up_sync(FULL, m[3].x, 1), __shfl_up_sync(FULL, m[3].y, 1));
    float ya[4], nya[4], nyr[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = cl + t;
      const float2 ml = t == 0 ? mL : m[t - 1];
      const float hl = t == 0 ? hl0 : hn[t - 1];
      float ca, r;
      edge_coef_r(ml, m[t], ca, r);
      nya[t] = ca;
      nyr[t] = __fmul_rn(r, sd.rdx2);
      const float v = __fmaf_rn(ca, eyA[t], -__fmul_rn(nyr[t], __fsub_rn(hn[t], hl)));
      const bool upd = i >= 1 && i < nx && ml.x >= 0.f && m[t].x >= 0.f;
      ya[t] = upd ? v : eyA[t];
      nmask |= upd ? 16u << t : 0u;
    }
    while (sa.j == j) {
      samples(sa.cs);
      march_source(ya, sa, cl, JA);
      sa = march_src_at(tm->src, ++kA, sr.y);
    }
    if constexpr (kFrames) {
      // E^{n+1}(j) into the intermediate frame (zone cells: the zone chain)
      bool keep = owner && j >= j0 && j < j1;
      for (int z = zr.x; z < zr.y; ++z) {
        const int4 zn = tm->zones[z];
        if (j >= zn.y && j < zn.w && cl < zn.z && cl + 4 > zn.x) keep = false;
      }
      if (keep) {
        const size_t off = (size_t)j * P + cl;
        st4(sd.exm + off, make_float4(xa[0], xa[1], xa[2], xa[3]));
        st4(sd.eym + off, make_float4(ya[0], ya[1], ya[2], ya[3]));
      }
    }
    // ---- carry to row j + 1
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      exc[t] = comp(cur.exn, t);
      hzp[t] = hn[t];
      mp[t] = m[t];
      xaP[t] = xa[t];
      yaP[t] = ya[t];
      cxa[t] = nxa[t];
      cxr[t] = nxr[t];
      cya[t] = nya[t];
      cyr[t] = nyr[t];
    }
    lmask = nmask;
    if constexpr (kRing == 0) cur = nxt;
  }
  // Launched after the model tiles of the same two steps (which it does not
  // read) with programmatic serialisation: it may start while they run, and
  // it does not complete before them, so the next launch sees both.
  pdl_wait();
}

using MarchFn = void (*)(const SimDev*, const TileWork*, const RunDev*, const TbMarchDev*, int, int, int);

// The row-marching kernel compiled for mb resident CTAs per SM, with loads
// in registers (ring 0) or staged through a ring of 2-4 rows, and with the
// background rows' materials taken without reading them (sparse: some
// simulation of the launch has a background material).
MarchFn march_fn(int mb, int ring, bool sparse) {
  if (mb == 3) return sparse ? yee_tb2m_kernel<3, 0, true> : yee_tb2m_kernel<3, 0, false>;
  switch (ring) {
    case 2: return sparse ? yee_tb2m_kernel<4, 2, true> : yee_tb2m_kernel<4, 2, false>;
    case 3: return sparse ? yee_tb2m_kernel<4, 3, true> : yee_tb2m_kernel<4, 3, false>;
    case 4: return sparse ? yee_tb2m_kernel<4, 4, true> : yee_tb2m_kernel<4, 4, false>;
    default: return sparse ? yee_tb2m_kernel<4, 0, true> : yee_tb2m_kernel<4, 0, false>;
  }
}
// Dynamic shared memory of a CTA of w warps (the ring of rows of each warp).
size_t march_smem(int ring, int w) { return ring > 0 ? (size_t)ring * (kMarchRingBytesPerRow / 4) * w : 0; }

// The form that also writes the intermediate E frame (sd.exm, sd.eym), for
// the plans the gradient's recomputation supports (else null).
MarchFn march_frames_fn(int mb, int ring, bool sparse) {
  if (mb == 3) return sparse ? yee_tb2m_kernel<3, 0, true, true> : yee_tb2m_kernel<3, 0, false, true>;
  if (mb != 4) return nullptr;
  if (ring == 0 && !sparse) return yee_tb2m_kernel<4, 0, false, true>;
  if (ring == 2) return sparse ? yee_tb2m_kernel<4, 2, true, true> : yee_tb2m_kernel<4, 2, false, true>;
  return nullptr;
}

}  // namespace
