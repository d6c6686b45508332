// Two time steps per launch (temporal blocking).  Included by fdtd.cu.
//
// A CTA stages a window of E^n, Hz^{n-1/2} and the cell materials of its
// output rectangle O = [X0, X1) x [Y0, Y1) in shared memory (cp.async, zero
// fill outside the arrays), then, in shared memory:
//   A.H  Hz^{n+1/2} on [X0-2, X1] x [Y0-2, Y1]                   (Eq. (5))
//   A.E  E^{n+1} on the edges of [X0-1, X1] x [Y0-1, Y1] + J^n    (Eq. (3))
//   (model tiles) [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2}      (Eq. (23))
//   B.H  Hz^{n+3/2} on [X0-1, X1-1] x [Y0-1, Y1-1]
//   B.E  E^{n+2} on the edges of O + J^{n+1}
//   (model tiles) [y; x~]^{n+2}
// and writes E^{n+2}, Hz^{n+3/2} of O.  Every cell depends only on values
// within two cells of it over two steps, so the window is O plus two cells
// (the interface values y^{n+1} of a model excepted).  Each model therefore
// gets a tile of its own whose O is its "zone" (the region grown by 3 cells)
// and which evaluates the model map between the sub-steps; ordinary tiles
// compute through zones with the plain update but do not write zone cells.
// Per step the DRAM traffic is about half that of the one-step kernel.

namespace {

constexpr int kTbW = 128;            // output columns of an ordinary tile (multiple of 4)
constexpr int kTbH = 32;             // output rows
constexpr int kTbSW = kTbW + 8;      // window columns [X0-4, X0+kTbW+4)
constexpr int kTbSH = kTbH + 4;      // window rows    [Y0-2, Y0+kTbH+2)
constexpr int kTbThreads = 256;
constexpr int kTbZoneMargin = 3;     // zone = region grown by this many cells
constexpr int kTbMaxRomN = 640;      // n + n_y limit for the in-CTA model step
constexpr size_t kTbSmemFields = sizeof(float) * (size_t)kTbSH * kTbSW * 5;

struct TbTile {
  int sim;
  int x0, x1, y0, y1;     // output rectangle O
  int rom;                // model instance owned (-1: ordinary tile)
  int zone_b, zone_e;     // ordinary tile: zones [b, e) in TbRun::zones to skip
  int src_b, src_e;       // source edges within the tile's E window
  int prb_b, prb_e;       // probes owned by the tile
  int scr;                // zone-chain tile: its window's scratch, in float4 units
};

struct TbRun {
  const int4* zones;        // x0, y0, x1, y1 of every zone
  const SrcEdge* src;       // per-tile source edges (TbTile ranges)
  const int* prb_idx;       // probe indices (TbTile ranges)
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz));
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// In-CTA model step: v = [s; h; 0] (ri.ld floats, 16-B aligned) staged in
// shared memory; rows split over warps.  The products and their order are
// those of rom_post_kernel's row-per-warp path, so both paths give the same
// bits.
__device__ void tb_rom_step(const RomInstDev& ri, const float* v, float* sout) {
  const unsigned FULL = 0xffffffffu;
  constexpr int R = 2;   // rows per warp at a time: their loads are in flight together
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float4* v4 = reinterpret_cast<const float4*>(v);
  const int l4 = ri.ld >> 2;
  for (int r0 = R * warp; r0 < ri.n; r0 += R * nw) {
    const float4* __restrict__ Mr[R];
    float acc[R];
#pragma unroll
    for (int u = 0; u < R; ++u) {   // rows past the end repeat the last row; not stored
      Mr[u] = reinterpret_cast<const float4*>(ri.M + (size_t)min(r0 + u, ri.n - 1) * ri.ld);
      acc[u] = 0.f;
    }
    for (int k = lane; k < l4; k += 32) {
      const float4 x = v4[k];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        const float4 m = Mr[u][k];
        acc[u] = fmaf(m.x, x.x, acc[u]);
        acc[u] = fmaf(m.y, x.y, acc[u]);
        acc[u] = fmaf(m.z, x.z, acc[u]);
        acc[u] = fmaf(m.w, x.w, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(FULL, acc[u], o);
      if (lane == 0 && r0 + u < ri.n) sout[r0 + u] = acc[u];
    }
  }
}

__global__ void __launch_bounds__(kTbThreads, 2)
yee_tb2_kernel(const SimDev* __restrict__ sims, const TbTile* __restrict__ tiles,
               const RomInstDev* __restrict__ insts, const RunDev* __restrict__ run,
               const TbRun* __restrict__ tb, int par, int c) {
  extern __shared__ float4 tb_smem4[];
  float* sEx = reinterpret_cast<float*>(tb_smem4);
  float* sEy = sEx + kTbSH * kTbSW;
  float* sHz = sEy + kTbSH * kTbSW;
  float2* sM = reinterpret_cast<float2*>(sHz + kTbSH * kTbSW);
  pdl_trigger();   // the row-marching kernel of the same two steps may start
  const TbTile tt = tiles[blockIdx.x];
  const SimDev sd = sims[tt.sim];
  const int nx = sd.nx, ny = sd.ny, P = sd.pitch;
  const float* __restrict__ ex = par ? sd.ex[1] : sd.ex[0];
  const float* __restrict__ ey = par ? sd.ey[1] : sd.ey[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  float* __restrict__ exo = par ? sd.ex[0] : sd.ex[1];
  float* __restrict__ eyo = par ? sd.ey[0] : sd.ey[1];
  float* __restrict__ hzo = par ? sd.hz[0] : sd.hz[1];
  const int X0 = tt.x0, X1 = tt.x1, Y0 = tt.y0, Y1 = tt.y1;
  const int wx = (X0 & ~3) - 4;   // window origin (16-B aligned column)
  const int wy = Y0 - 2;
  const int tid = threadIdx.x;
  // ---- stage the window
  {
    constexpr int q4 = kTbSW / 4;
    for (int e = tid; e < kTbSH * q4; e += kTbThreads) {
      const int r = e / q4, q = e % q4;
      const int j = wy + r, i = wx + 4 * q;
      const bool ok = (j >= 0) && (j <= ny) && (i >= 0) && (i + 3 < P);
      const size_t off = ok ? (size_t)j * P + i : 0;
      cp_async16(sEx + r * kTbSW + 4 * q, ex + off, ok);
      cp_async16(sEy + r * kTbSW + 4 * q, ey + off, ok);
      cp_async16(sHz + r * kTbSW + 4 * q, hz + off, ok);
      cp_async16(sM + r * kTbSW + 4 * q, sd.mat + off, ok);
      cp_async16(sM + r * kTbSW + 4 * q + 2, sd.mat + off + 2, ok);
    }
    cp_async_wait_all();
    __syncthreads();
  }
  auto S = [&](int i, int j) { return (j - wy) * kTbSW + (i - wx); };
  // Cells outside the grid are marked dead (their edges are PEC or outside).
  if (wx < 0 || wx + kTbSW > nx || wy < 0 || wy + kTbSH > ny) {
    for (int e = tid; e < kTbSH * kTbSW; e += kTbThreads) {
      const int i = wx + e % kTbSW, j = wy + e / kTbSW;
      if (i < 0 || i >= nx || j < 0 || j >= ny) sM[e].x = -1.f;
    }
    __syncthreads();
  }
  // Both sub-steps update the whole window (H: rows 0..SH-2, E: rows 1..SH-1)
  // in float4 units; values within 3 cells of the window edge use neighbours
  // outside the window and are wrong, but no output depends on them (the
  // outputs are 4 columns and 2 rows inside the window).
  constexpr int q4 = kTbSW / 4;
  auto h_update = [&]() {
    for (int u = tid; u < (kTbSH - 1) * q4; u += kTbThreads) {
      const int s = (u / q4) * kTbSW + 4 * (u % q4);
      const float4 e0 = ld4(sEx + s), e1 = ld4(sEx + s + kTbSW), yv = ld4(sEy + s);
      float4 h = ld4(sHz + s);
      const float4 ma = ld4(reinterpret_cast<const float*>(sM + s));
      const float4 mb = ld4(reinterpret_cast<const float*>(sM + s + 2));
      const float yA[5] = {yv.x, yv.y, yv.z, yv.w, sEy[s + 4]};
      const float mx[4] = {ma.x, ma.z, mb.x, mb.z};
      float hn[4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        hn[t] = mx[t] >= 0.f ? __fsub_rn(__fmaf_rn(sd.chx, __fsub_rn(comp(e1, t), comp(e0, t)), comp(h, t)),
                                          __fmul_rn(sd.chy, __fsub_rn(yA[t + 1], yA[t])))
                            : 0.f;
      st4(sHz + s, make_float4(hn[0], hn[1], hn[2], hn[3]));
    }
  };
  auto e_update = [&]() {
    for (int u = tid; u < (kTbSH - 1) * q4; u += kTbThreads) {
      const int s = (u / q4 + 1) * kTbSW + 4 * (u % q4);
      const float4 h = ld4(sHz + s), hd = ld4(sHz + s - kTbSW);
      const float hL = sHz[s - 1];
      float4 xv = ld4(sEx + s), yv = ld4(sEy + s);
      const float4 ma = ld4(reinterpret_cast<const float*>(sM + s));
      const float4 mb = ld4(reinterpret_cast<const float*>(sM + s + 2));
      const float4 da = ld4(reinterpret_cast<const float*>(sM + s - kTbSW));
      const float4 db = ld4(reinterpret_cast<const float*>(sM + s - kTbSW + 2));
      const float2 mL = sM[s - 1];
      const float2 m[4] = {make_float2(ma.x, ma.y), make_float2(ma.z, ma.w), make_float2(mb.x, mb.y),
                           make_float2(mb.z, mb.w)};
      const float2 md[4] = {make_float2(da.x, da.y), make_float2(da.z, da.w), make_float2(db.x, db.y),
                            make_float2(db.z, db.w)};
      float xo[4], yo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float v = comp(xv, t);
        if (md[t].x >= 0.f && m[t].x >= 0.f) {
          float ca, cb;
          edge_coef(md[t], m[t], ca, cb);
          v = __fmaf_rn(ca, v, __fmul_rn(__fmul_rn(cb, sd.rdy), __fsub_rn(comp(h, t), comp(hd, t))));
        }
        xo[t] = v;
        const float2 ml = t == 0 ? mL : m[t - 1];
        const float hl = t == 0 ? hL : comp(h, t - 1);
        float w = comp(yv, t);
        if (ml.x >= 0.f && m[t].x >= 0.f) {
          float ca, cb;
          edge_coef(ml, m[t], ca, cb);
          w = __fmaf_rn(ca, w, -__fmul_rn(__fmul_rn(cb, sd.rdx), __fsub_rn(comp(h, t), hl)));
        }
        yo[t] = w;
      }
      st4(sEx + s, make_float4(xo[0], xo[1], xo[2], xo[3]));
      st4(sEy + s, make_float4(yo[0], yo[1], yo[2], yo[3]));
    }
  };
  auto sources = [&](int ia, int ib, int ja, int jb, long long n) {
    for (int e = tt.src_b + tid; e < tt.src_e; e += kTbThreads) {
      const SrcEdge se = tb->src[e];
      if (se.i < ia || se.i > ib || se.j < ja || se.j > jb) continue;
      const int s = S(se.i, se.j);
      float ca, cb;
      edge_coef(se.comp == 0 ? sM[s - kTbSW] : sM[s - 1], sM[s], ca, cb);
      float& d = (se.comp == 0 ? sEx : sEy)[s];
      d = __fsub_rn(d, __fmul_rn(cb, run->waves[se.src][n]));
    }
  };
  auto probes = [&](long long n) {
    for (int e = tt.prb_b + tid; e < tt.prb_e; e += kTbThreads) {
      const int p = tb->prb_idx[e];
      const int cell = run->probe_cell[p];
      run->probe_out[n * run->nprobe + p] = sHz[S(cell % P, cell / P)];
    }
  };
  // model state staging (model tiles): s_state[b] = [s; h; 0], ri.ld floats
  __shared__ __align__(16) float s_state[2][kTbMaxRomN];
  RomInstDev ri{};
  if (tt.rom >= 0) {
    ri = insts[tt.rom];
    const float* st = par ? ri.state[1] : ri.state[0];
    for (int k = tid; k < ri.ld; k += kTbThreads) {
      s_state[0][k] = k < ri.n ? st[k] : 0.f;
      s_state[1][k] = 0.f;
    }
  }
  auto rom_phase = [&](int from) {   // s_state[from] -> s_state[1-from], y into sEx/sEy
    float* hv = s_state[from] + ri.n;
    for (int k = tid; k < ri.ny; k += kTbThreads) {
      const int cell = ri.h_cell[k];
      hv[k] = sHz[S(cell % P, cell / P)];
    }
    __syncthreads();
    tb_rom_step(ri, s_state[from], s_state[1 - from]);
    __syncthreads();
    for (int k = tid; k < ri.ny; k += kTbThreads) {
      const int code = ri.y_edge[k];
      const int off = code & 0x3fffffff;
      (code >> 30 ? sEy : sEx)[S(off % P, off / P)] = s_state[1 - from][k];
    }
    __syncthreads();
  };
  const long long n0 = run->base + 2 * (long long)c;
  // ---- step n
  h_update();
  __syncthreads();
  probes(n0);
  e_update();
  __syncthreads();
  sources(X0 - 1, X1, Y0 - 1, Y1, n0);
  __syncthreads();
  if (tt.rom >= 0) rom_phase(0);
  // ---- step n+1
  h_update();
  __syncthreads();
  probes(n0 + 1);
  e_update();
  __syncthreads();
  sources(X0, X1 - 1, Y0, Y1 - 1, n0 + 1);
  __syncthreads();
  if (tt.rom >= 0) {
    rom_phase(1);
    float* so = par ? ri.state[0] : ri.state[1];
    for (int k = tid; k < ri.n; k += kTbThreads) so[k] = s_state[0][k];
  }
  // ---- write O (ordinary tiles skip zone cells)
  if (tt.rom < 0 && tt.zone_b == tt.zone_e && ((X1 - X0) & 3) == 0) {
    const int w4 = (X1 - X0) >> 2;
    for (int e = tid; e < w4 * (Y1 - Y0); e += kTbThreads) {
      const int i = X0 + 4 * (e % w4), j = Y0 + e / w4;
      const int s = S(i, j);
      const size_t off = (size_t)j * P + i;
      st4(hzo + off, ld4(sHz + s));
      st4(exo + off, ld4(sEx + s));
      st4(eyo + off, ld4(sEy + s));
    }
  } else {
    const int w = X1 - X0;
    for (int e = tid; e < w * (Y1 - Y0); e += kTbThreads) {
      const int i = X0 + e % w, j = Y0 + e / w;
      bool own = true;
      for (int z = tt.zone_b; z < tt.zone_e; ++z) {
        const int4 zn = tb->zones[z];
        if (i >= zn.x && i < zn.z && j >= zn.y && j < zn.w) own = false;
      }
      if (!own) continue;
      const int s = S(i, j);
      const size_t off = (size_t)j * P + i;
      hzo[off] = sHz[s];
      exo[off] = sEx[s];
      eyo[off] = sEy[s];
    }
  }
}

// ---- two-step path with the model maps stepped outside the tile ----------
// For models whose map is shared by many simulations (or any model, on
// request), the zone tile is split in two launches around the map of
// Eq. (23), so that the maps of all instances sharing [P | Q] run as one GEMM
// and a large map is spread over many CTAs:
//   half 0  stage the window, A.H (probes n), A.E (+ J^n); h^{n+1/2} into the
//           tail of the model's input vector [s^n; h]; the window to scratch;
//   map     s^{n+1} = [P | Q] [s^n; h^{n+1/2}]                 (rom_chain_kernel)
//   half 1  restore the window, y^{n+1} onto the interface edges, B.H
//           (probes n+1), B.E (+ J^{n+1}); h^{n+3/2} into [s^{n+1}; h]; write O;
//   map     s^{n+2} = [P | Q] [s^{n+1}; h^{n+3/2}], y^{n+2} onto the output
//           interface edges (after half 1 wrote O).
// The window holds what O depends on: rows Y0-2 .. Y1+1 and the float4
// groups from the aligned column X0-4 to past X1+1, plus one spare group read
// by the last group's Hz update, packed with a row stride of SW = 4 SW4
// floats.  Every update is yee_tb2_kernel's operation sequence and the map is
// rom_post_kernel's, so the result is the fused model tile's bit for bit.

__host__ __device__ __forceinline__ int zone_sw4(int x0, int x1) { return (x1 - ((x0 & ~3) - 4) + 9) / 4 + 1; }
__host__ __device__ __forceinline__ int zone_rows(int y0, int y1) { return y1 - y0 + 4; }

template <int kHalf>
__global__ void __launch_bounds__(kTbThreads, 2)
zone_step_kernel(const SimDev* __restrict__ sims, const TbTile* __restrict__ tiles,
                 const RomInstDev* __restrict__ insts, const RunDev* __restrict__ run,
                 const TbRun* __restrict__ tb, float* __restrict__ scratch, int par, int c) {
  extern __shared__ float4 zs_smem4[];
  const TbTile tt = tiles[blockIdx.x];
  const SimDev sd = sims[tt.sim];
  const RomInstDev ri = insts[tt.rom];
  const int nx = sd.nx, ny = sd.ny, P = sd.pitch;
  const int X0 = tt.x0, X1 = tt.x1, Y0 = tt.y0, Y1 = tt.y1;
  const int wx = (X0 & ~3) - 4, wy = Y0 - 2;
  const int SW4 = zone_sw4(X0, X1), SW = 4 * SW4, nR = zone_rows(Y0, Y1), NF = nR * SW;
  float* sEx = reinterpret_cast<float*>(zs_smem4);
  float* sEy = sEx + NF;
  float* sHz = sEy + NF;
  float2* sM = reinterpret_cast<float2*>(sHz + NF);
  float* __restrict__ scr = scratch + 4 * (size_t)tt.scr;   // 3 NF floats: Ex, Ey, Hz after A
  const float* __restrict__ ex = par ? sd.ex[1] : sd.ex[0];
  const float* __restrict__ ey = par ? sd.ey[1] : sd.ey[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  const int tid = threadIdx.x;
  // ---- stage the window (half 0) or restore it (half 1), and the materials
  for (int e = tid; e < nR * SW4; e += kTbThreads) {
    const int r = e / SW4, q = e - r * SW4;
    const int j = wy + r, i = wx + 4 * q;
    const bool ok = (j >= 0) && (j <= ny) && (i >= 0) && (i + 3 < P);
    const size_t off = ok ? (size_t)j * P + i : 0;
    if (kHalf == 0) {
      cp_async16(sEx + r * SW + 4 * q, ex + off, ok);
      cp_async16(sEy + r * SW + 4 * q, ey + off, ok);
      cp_async16(sHz + r * SW + 4 * q, hz + off, ok);
    }
    cp_async16(sM + r * SW + 4 * q, sd.mat + off, ok);
    cp_async16(sM + r * SW + 4 * q + 2, sd.mat + off + 2, ok);
  }
  if (kHalf == 1)
    for (int e = tid; e < 3 * NF / 4; e += kTbThreads) cp_async16(sEx + 4 * e, scr + 4 * e, true);
  cp_async_wait_all();
  __syncthreads();
  auto S = [&](int i, int j) { return (j - wy) * SW + (i - wx); };
  if (wx < 0 || wx + SW > nx || wy < 0 || wy + nR > ny) {
    for (int e = tid; e < NF; e += kTbThreads) {
      const int i = wx + e % SW, j = wy + e / SW;
      if (i < 0 || i >= nx || j < 0 || j >= ny) sM[e].x = -1.f;
    }
    __syncthreads();
  }
  const int q4 = SW4 - 1;   // groups updated (the spare one is only read)
  auto h_update = [&]() {
    for (int u = tid; u < (nR - 1) * q4; u += kTbThreads) {
      const int s = (u / q4) * SW + 4 * (u % q4);
      const float4 e0 = ld4(sEx + s), e1 = ld4(sEx + s + SW), yv = ld4(sEy + s);
      float4 h = ld4(sHz + s);
      const float4 ma = ld4(reinterpret_cast<const float*>(sM + s));
      const float4 mb = ld4(reinterpret_cast<const float*>(sM + s + 2));
      const float yA[5] = {yv.x, yv.y, yv.z, yv.w, sEy[s + 4]};
      const float mx[4] = {ma.x, ma.z, mb.x, mb.z};
      float hn[4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        hn[t] = mx[t] >= 0.f ? __fsub_rn(__fmaf_rn(sd.chx, __fsub_rn(comp(e1, t), comp(e0, t)), comp(h, t)),
                                          __fmul_rn(sd.chy, __fsub_rn(yA[t + 1], yA[t])))
                            : 0.f;
      st4(sHz + s, make_float4(hn[0], hn[1], hn[2], hn[3]));
    }
  };
  auto e_update = [&]() {
    for (int u = tid; u < (nR - 1) * q4; u += kTbThreads) {
      const int s = (u / q4 + 1) * SW + 4 * (u % q4);
      const float4 h = ld4(sHz + s), hd = ld4(sHz + s - SW);
      const float hL = sHz[s - 1];
      float4 xv = ld4(sEx + s), yv = ld4(sEy + s);
      const float4 ma = ld4(reinterpret_cast<const float*>(sM + s));
      const float4 mb = ld4(reinterpret_cast<const float*>(sM + s + 2));
      const float4 da = ld4(reinterpret_cast<const float*>(sM + s - SW));
      const float4 db = ld4(reinterpret_cast<const float*>(sM + s - SW + 2));
      const float2 mL = sM[s - 1];
      const float2 m[4] = {make_float2(ma.x, ma.y), make_float2(ma.z, ma.w), make_float2(mb.x, mb.y),
                           make_float2(mb.z, mb.w)};
      const float2 md[4] = {make_float2(da.x, da.y), make_float2(da.z, da.w), make_float2(db.x, db.y),
                            make_float2(db.z, db.w)};
      float xo[4], yo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float v = comp(xv, t);
        if (md[t].x >= 0.f && m[t].x >= 0.f) {
          float ca, cb;
          edge_coef(md[t], m[t], ca, cb);
          v = __fmaf_rn(ca, v, __fmul_rn(__fmul_rn(cb, sd.rdy), __fsub_rn(comp(h, t), comp(hd, t))));
        }
        xo[t] = v;
        const float2 ml = t == 0 ? mL : m[t - 1];
        const float hl = t == 0 ? hL : comp(h, t - 1);
        float w = comp(yv, t);
        if (ml.x >= 0.f && m[t].x >= 0.f) {
          float ca, cb;
          edge_coef(ml, m[t], ca, cb);
          w = __fmaf_rn(ca, w, -__fmul_rn(__fmul_rn(cb, sd.rdx), __fsub_rn(comp(h, t), hl)));
        }
        yo[t] = w;
      }
      st4(sEx + s, make_float4(xo[0], xo[1], xo[2], xo[3]));
      st4(sEy + s, make_float4(yo[0], yo[1], yo[2], yo[3]));
    }
  };
  auto sources = [&](int ia, int ib, int ja, int jb, long long n) {
    for (int e = tt.src_b + tid; e < tt.src_e; e += kTbThreads) {
      const SrcEdge se = tb->src[e];
      if (se.i < ia || se.i > ib || se.j < ja || se.j > jb) continue;
      const int s = S(se.i, se.j);
      float ca, cb;
      edge_coef(se.comp == 0 ? sM[s - SW] : sM[s - 1], sM[s], ca, cb);
      float& d = (se.comp == 0 ? sEx : sEy)[s];
      d = __fsub_rn(d, __fmul_rn(cb, run->waves[se.src][n]));
    }
  };
  auto probes = [&](long long n) {
    for (int e = tt.prb_b + tid; e < tt.prb_e; e += kTbThreads) {
      const int p = tb->prb_idx[e];
      const int cell = run->probe_cell[p];
      run->probe_out[n * run->nprobe + p] = sHz[S(cell % P, cell / P)];
    }
  };
  const long long n0 = run->base + 2 * (long long)c;
  if constexpr (kHalf == 0) {
    h_update();
    __syncthreads();
    probes(n0);
    e_update();
    __syncthreads();
    sources(X0 - 1, X1, Y0 - 1, Y1, n0);
    __syncthreads();
    float* __restrict__ sin = par ? ri.state[1] : ri.state[0];
    for (int k = tid; k < ri.ny; k += kTbThreads) {
      const int cell = ri.h_cell[k];
      sin[ri.n + k] = sHz[S(cell % P, cell / P)];
    }
    for (int e = tid; e < 3 * NF / 4; e += kTbThreads) st4(scr + 4 * e, ld4(sEx + 4 * e));
  } else {
    for (int k = tid; k < ri.ny; k += kTbThreads) {   // y^{n+1}
      const int code = ri.y_edge[k];
      const int off = code & 0x3fffffff;
      (code >> 30 ? sEy : sEx)[S(off % P, off / P)] = ri.state_mid[k];
    }
    __syncthreads();
    if (sd.exm) {   // E^{n+1} of the zone into the intermediate frame
      const int w = X1 - X0;
      for (int e = tid; e < w * (Y1 - Y0); e += kTbThreads) {
        const int i = X0 + e % w, j = Y0 + e / w;
        const size_t off = (size_t)j * P + i;
        sd.exm[off] = sEx[S(i, j)];
        sd.eym[off] = sEy[S(i, j)];
      }
    }
    h_update();
    __syncthreads();
    probes(n0 + 1);
    e_update();
    __syncthreads();
    sources(X0, X1 - 1, Y0, Y1 - 1, n0 + 1);
    __syncthreads();
    for (int k = tid; k < ri.ny; k += kTbThreads) {   // h^{n+3/2}
      const int cell = ri.h_cell[k];
      ri.state_mid[ri.n + k] = sHz[S(cell % P, cell / P)];
    }
    float* __restrict__ exo = par ? sd.ex[0] : sd.ex[1];
    float* __restrict__ eyo = par ? sd.ey[0] : sd.ey[1];
    float* __restrict__ hzo = par ? sd.hz[0] : sd.hz[1];
    const int w = X1 - X0;
    for (int e = tid; e < w * (Y1 - Y0); e += kTbThreads) {
      const int i = X0 + e % w, j = Y0 + e / w;
      const int s = S(i, j);
      const size_t off = (size_t)j * P + i;
      hzo[off] = sHz[s];
      exo[off] = sEx[s];
      eyo[off] = sEy[s];
    }
  }
}

// Eq. (23) for the models of the zone chain: s_out = [P | Q] [s_in; h], the
// input vector read whole from the model's state buffer (its h part placed
// there by zone_step_kernel).  which = 0: state[in] -> state_mid (s^{n+1});
// which = 1: state_mid -> state[out] (s^{n+2}) and y^{n+2} onto the output
// interface edges.  Blocks [0, nwork) step single models one row per warp,
// the rest the GEMM tiles of shared maps; both with rom_post_kernel's
// operations in its order.
__global__ void __launch_bounds__(kRomRowsPerCta * 32)
rom_chain_kernel(const SimDev* __restrict__ sims, const RomInstDev* __restrict__ insts,
                 const RomWork* __restrict__ work, int nwork, const GemmGroupDev* __restrict__ groups,
                 const GemmWork* __restrict__ gwork, const int* __restrict__ ginst, int par, int which) {
  extern __shared__ float4 rc_smem4[];
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto in_of = [&](const RomInstDev& ri) -> const float* {
    return which ? ri.state_mid : (par ? ri.state[1] : ri.state[0]);
  };
  auto out_of = [&](const RomInstDev& ri) -> float* { return which ? (par ? ri.state[0] : ri.state[1]) : ri.state_mid; };
  auto scatter = [&](const RomInstDev& ri, int r, float v) {
    if (which && r < ri.ny) {
      const SimDev* sd = sims + ri.sim;
      const int code = ri.y_edge[r];
      float* base = (code >> 30) ? (par ? sd->ey[0] : sd->ey[1]) : (par ? sd->ex[0] : sd->ex[1]);
      base[code & 0x3fffffff] = v;
    }
  };
  if ((int)blockIdx.x < nwork) {
    const RomWork w = work[blockIdx.x];
    const RomInstDev ri = insts[w.inst];
    const float* __restrict__ in = in_of(ri);
    float* v = reinterpret_cast<float*>(rc_smem4);
    for (int k = tid; 4 * k < ri.ld; k += blockDim.x) async_copy16(v + 4 * k, in + 4 * k);
    async_wait_all();
    __syncthreads();
    const int r = w.row0 + warp;
    if (r >= w.row1) return;
    const float4* __restrict__ Mr = reinterpret_cast<const float4*>(ri.M + (size_t)r * ri.ld);
    const int l4 = ri.ld >> 2;
    float acc = 0.f;
    for (int k = lane; k < l4; k += 32) {
      const float4 m = Mr[k];
      const float4 x = rc_smem4[k];
      acc = fmaf(m.x, x.x, acc);
      acc = fmaf(m.y, x.y, acc);
      acc = fmaf(m.z, x.z, acc);
      acc = fmaf(m.w, x.w, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) {
      out_of(ri)[r] = acc;
      scatter(ri, r, acc);
    }
    return;
  }
  const GemmWork gw = gwork[blockIdx.x - nwork];
  const GemmGroupDev g = groups[gw.group];
  __shared__ int s_inst[32];
  const int nc = min(32, g.B - gw.c0);
  const int ld = g.ld;
  if (tid < nc) s_inst[tid] = ginst[g.inst_off + gw.c0 + tid];
  __syncthreads();
  float* panel = reinterpret_cast<float*>(rc_smem4);   // [col][k], ld floats per column
  for (int col = warp; col < 32; col += kRomRowsPerCta) {
    float* pc = panel + (size_t)col * ld;
    if (col < nc) {
      const float* __restrict__ in = in_of(insts[s_inst[col]]);
      for (int k = lane; 4 * k < ld; k += 32) async_copy16(pc + 4 * k, in + 4 * k);
    } else {
      for (int k = lane; k < ld; k += 32) pc[k] = 0.f;
    }
  }
  async_wait_all();
  __syncthreads();
  auto rows = [&](auto rpw_c) {
    constexpr int RPW = decltype(rpw_c)::value;
    const int rb = gw.r0 + RPW * warp;
    if (rb >= g.n) return;
    const float4* Mr[RPW];
#pragma unroll
    for (int i = 0; i < RPW; ++i)   // rows past the end repeat the last row; not stored
      Mr[i] = reinterpret_cast<const float4*>(g.M + (size_t)min(rb + i, g.n - 1) * ld);
    float res[RPW];
    gemm_exact_rows<RPW>(Mr, ld >> 2, panel, ld, lane, res);
    if (lane >= nc) return;
    const RomInstDev ri = insts[s_inst[lane]];
    float* __restrict__ so = out_of(ri);
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
      const int r = rb + i;
      if (r < g.n) {
        so[r] = res[i];
        scatter(ri, r, res[i]);
      }
    }
  };
  if (g.rpw == 2) rows(std::integral_constant<int, 2>{});
  else rows(std::integral_constant<int, 1>{});
}

}  // namespace
