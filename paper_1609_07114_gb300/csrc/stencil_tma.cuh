// Bulk-copy form of the fused coarse step: the rows a warp needs are staged
// in shared memory by the TMA engine (cp.async.bulk, completion on one
// mbarrier per ring slot), kTmaDepth rows ahead of the row being computed,
// so a warp keeps about 3 x 2.6 KB of loads in flight without holding them
// in registers.  The arithmetic is stencil_row, shared with the
// register-prefetch kernel (identical results).
//
// Shared memory per warp: kTmaDepth slots of one row each,
//   Ex(j+1), Ey(j), Hz(j): columns [c0 - 4, c0 + 132) (136 floats each),
//   mat(j): columns [c0 - 2, c0 + 128) (130 float2),
// a window clipped to [c0, ...) when c0 = 0 and to [..., c0 + 128) when
// c0 + 132 passes the row pitch (the extra column c0 + 128 is then not an
// edge of the grid).  Every window starts on a 16-byte boundary and has a
// multiple of 16 bytes, as bulk copies require.  Strip rows whose cells are
// all background skip the material copy.
#pragma once

// (included inside the anonymous namespace of fdtd.cu)

constexpr int kTmaDepth = 4;
constexpr int kTmaSlotFloats = 672;                        // 2688 B
constexpr int kTmaEx = 0, kTmaEy = 136, kTmaHz = 272, kTmaMat = 408;
constexpr int kTmaWarps = kCtaCols / 128;
constexpr int kTmaRingBytes = kTmaWarps * kTmaDepth * kTmaSlotFloats * 4;
constexpr int kTmaSmem = kTmaRingBytes + kTmaWarps * kTmaDepth * 8;
// try_wait polls before a wait is declared lost (each poll may suspend the
// thread for a hardware-chosen time; the limit is far beyond any copy).
constexpr unsigned kTmaSpinLimit = 1u << 24;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait; false if the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = kTmaSpinLimit) {
  for (unsigned k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Self-test of the failure path of the bounded waits: every thread waits on
// a barrier that nothing arrives at (no copy is ever issued to it), gives up
// after `limit` polls and reports through the status word, as the stencil's
// waits do.
__global__ void wait_selftest_kernel(unsigned* status, unsigned limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u, limit);
  if (__any_sync(0xffffffffu, !ok) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

__global__ void __launch_bounds__(kCtaCols / 4, 4)
yee_step_tma_kernel(const SimDev* __restrict__ sims, const TileWork* __restrict__ work,
                    const RunDev* __restrict__ run, int par, int c) {
  extern __shared__ __align__(128) unsigned char tma_smem[];
  const TileWork tw = work[blockIdx.x];
  const SimDev sd = sims[tw.sim];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = tw.x0 + warp * 128;
  const int nx = sd.nx, P = sd.pitch;
  const float* __restrict__ ex = par ? sd.ex[1] : sd.ex[0];
  const float* __restrict__ ey = par ? sd.ey[1] : sd.ey[0];
  const float* __restrict__ hz = par ? sd.hz[1] : sd.hz[0];
  float* __restrict__ exo = par ? sd.ex[0] : sd.ex[1];
  float* __restrict__ eyo = par ? sd.ey[0] : sd.ey[1];
  float* __restrict__ hzo = par ? sd.hz[0] : sd.hz[1];
  const float2* __restrict__ mat = sd.mat;
  float* ring = reinterpret_cast<float*>(tma_smem) + warp * kTmaDepth * kTmaSlotFloats;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tma_smem + kTmaRingBytes) + warp * kTmaDepth;
  if (c0 < nx) {
    const int cl = c0 + 4 * lane;
    const int j0 = tw.y0, j1 = tw.y1;
    const int js = j0 > 0 ? j0 - 1 : 0;
    const bool halo = (lane == 0) && (c0 > 0);
    // global windows of one row (columns), their byte counts and their
    // offsets (floats) inside a slot
    const int fs = c0 > 0 ? c0 - 4 : c0;
    const int fe = (c0 + 132 <= P) ? c0 + 132 : c0 + 128;
    const int ms = c0 > 0 ? c0 - 2 : c0;
    const unsigned fbytes = 4u * (unsigned)(fe - fs);
    const unsigned mbytes = 8u * (unsigned)(c0 + 128 - ms);
    const int fo = fs - (c0 - 4);
    const int mo = 2 * (ms - (c0 - 2));
    RowCarry<4> cy;
    uint32_t fw;
    BgCoef bc;
    stencil_start<4>(sd, ex, js, cl, c0, lane, halo, cy, fw, bc);
    if (lane == 0) {
      for (int s = 0; s < kTmaDepth; ++s) mbar_init(&bars[s], 1);
      mbar_fence_init();
    }
    __syncwarp();
    // lane 0 only: stage row jj into its slot
    auto issue = [&](int jj, bool dn) {
      const int s = (jj - js) % kTmaDepth;
      float* slot = ring + s * kTmaSlotFloats;
      const size_t row = (size_t)jj * P;
      mbar_expect_tx(&bars[s], 3u * fbytes + (dn ? mbytes : 0u));
      bulk_copy_g2s(slot + kTmaEx + fo, ex + row + P + fs, fbytes, &bars[s]);
      bulk_copy_g2s(slot + kTmaEy + fo, ey + row + fs, fbytes, &bars[s]);
      bulk_copy_g2s(slot + kTmaHz + fo, hz + row + fs, fbytes, &bars[s]);
      if (dn) bulk_copy_g2s(slot + kTmaMat + mo, mat + row + ms, mbytes, &bars[s]);
    };
#pragma unroll 1
    for (int k = 0; k < kTmaDepth; ++k) {
      const int jj = js + k;
      const bool dn = strip_dense(fw, js, jj < j1 ? jj : js);
      if (lane == 0 && jj < j1) issue(jj, dn);
    }
    const float2 bg = sd.mbg;
    bool dcur = strip_dense(fw, js, js), dprev = true;
    int j = js;
    for (; j < j1; ++j) {
      const int k = j - js, s = k % kTmaDepth;
      const float* slot = ring + s * kTmaSlotFloats;
      const bool ok = mbar_wait(&bars[s], (unsigned)(k / kTmaDepth) & 1u);
      if (__any_sync(0xffffffffu, !ok)) break;
      RowIn<4> cur;
      cur.exn = *reinterpret_cast<const float4*>(slot + kTmaEx + 4 + 4 * lane);
      cur.eyv = *reinterpret_cast<const float4*>(slot + kTmaEy + 4 + 4 * lane);
      cur.hzv = *reinterpret_cast<const float4*>(slot + kTmaHz + 4 + 4 * lane);
      if (dcur) {
        cur.m4[0] = *reinterpret_cast<const float4*>(slot + kTmaMat + 4 + 8 * lane);
        cur.m4[1] = *reinterpret_cast<const float4*>(slot + kTmaMat + 8 + 8 * lane);
      } else {
        cur.m4[0] = cur.m4[1] = make_float4(bg.x, bg.y, bg.x, bg.y);
      }
      cur.eyR = (lane == 31 && c0 + 128 <= nx) ? slot[kTmaEy + 132] : 0.f;
      if (halo) {
        cur.exLn = slot[kTmaEx + 3];
        cur.eyL = slot[kTmaEy + 3];
        cur.hzL = slot[kTmaHz + 3];
        cur.mL = dcur ? *reinterpret_cast<const float2*>(slot + kTmaMat + 2) : bg;
      } else {
        cur.exLn = cur.eyL = cur.hzL = 0.f;
        cur.mL = make_float2(-1.f, 0.f);
      }
      // every lane has read the slot: refill it with row j + kTmaDepth
      __syncwarp();
      const int jn = j + kTmaDepth;
      const bool dnn = strip_dense(fw, js, jn < j1 ? jn : j);
      if (lane == 0 && jn < j1) {
        fence_proxy_async_smem();
        issue(jn, dnn);
      }
      const bool dn = strip_dense(fw, js, j + 1 < j1 ? j + 1 : j);
      stencil_row<4>(sd, cur, cy, j, j0, cl, nx, lane, halo, dcur, dprev, bc, (size_t)j * P, hzo, exo, eyo);
      dprev = dcur;
      dcur = dn;
    }
    if (j < j1) {
      // a wait gave up: report it, then wait (bounded) for the copies still
      // in flight into this warp's slots before the CTA may exit
      if (lane == 0) {
        atomicOr(run->status, 1u);
        const int last = min(j1, j + kTmaDepth);
        for (int jj = j; jj < last; ++jj) {
          const int k = jj - js;
          mbar_wait(&bars[k % kTmaDepth], (unsigned)(k / kTmaDepth) & 1u);
        }
      }
      __syncwarp();
    }
  }
  stencil_sources(run, c, mat, P, exo, eyo);
}
