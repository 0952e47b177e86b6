// A5: brute-force incoherent dedispersion (Sec. 2.2.2, delays of Eq. 1)
//
//   D[d][t] = sum_{c=0}^{nchan-1} y[c][t + delay[d][c]],   0 <= t < T,
//
// over the substituted, bandpass-corrected series y written by the A3/A4
// kernel (FP32; exact small integers for 8-bit data).
//
// Work decomposition.  A CTA owns a tile of consecutive DM trials (up to 8
// groups of K) x TT = 32 S output samples; warp w owns group w, lane l owns
// the S consecutive outputs t0 + l S .. t0 + l S + S - 1 of each of the K DMs.
// The CTA walks the channels in order, NC per pipeline stage: for every
// channel one elected thread copies the samples the tile needs,
// [t0 + delay[d_first][c], t0 + TT + delay[d_last][c]) rounded out to 16 B,
// from global into shared memory with cp.async.bulk, completing on an
// mbarrier (NSTAGE stages in flight).  The consumer warps then load, per lane,
// a register window of S + spread + 4 consecutive samples with 128-bit shared
// loads and add it into the K x S accumulators at each DM's offset inside the
// window.  The offsets are warp-uniform run-time values, so each DM selects an
// unrolled add sequence through a switch over 0..OMAX: every sample loaded
// from shared memory feeds up to K adds from registers.  Each (d, t) adds its
// channels in index order in FP32.
//
// The epilogue writes D (FP32, or int32 for 8-bit data, exact) and per
// (DM, time tile) sums of D and D^2 for the series statistics of A6.
#include <cstdint>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = 8;
constexpr int kNC = 4;                 // channels per pipeline stage
constexpr int kStages = 4;             // pipeline depth
constexpr long long kSpinLimit = 1LL << 24;  // bounded mbarrier waits

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <int S, int L, int O>
__device__ __forceinline__ void add_at(float (&acc)[S], const float (&w)[L]) {
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] += w[O + s];
}

#define TP_CASE(o)                                       \
  case (o):                                              \
    if constexpr ((o) <= OMAX) add_at<S, L, (o)>(acc, w); \
    break;
#define TP_CASE8(b) \
  TP_CASE(b + 0) TP_CASE(b + 1) TP_CASE(b + 2) TP_CASE(b + 3) TP_CASE(b + 4) TP_CASE(b + 5) TP_CASE(b + 6) TP_CASE(b + 7)

// acc[s] += w[o + s] for a warp-uniform o in [0, OMAX] (OMAX <= 63).
template <int S, int L, int OMAX>
__device__ __forceinline__ void add_shifted(int o, float (&acc)[S], const float (&w)[L]) {
  static_assert(OMAX < 64, "offset range");
  switch (o) {
    TP_CASE8(0) TP_CASE8(8) TP_CASE8(16) TP_CASE8(24) TP_CASE8(32) TP_CASE8(40) TP_CASE8(48) TP_CASE8(56)
    default: break;
  }
}
#undef TP_CASE8
#undef TP_CASE

template <int K, int S, int OMAX>
struct Shape {
  static constexpr int TT = 32 * S;                        // output samples per tile
  static constexpr int L = ((S + OMAX + 1) + 3) / 4 * 4;   // register window
  static constexpr int ROW = (TT + kMaxOverhang + OMAX + 8 + 31) / 32 * 32;  // staged floats per channel
  static constexpr size_t smem = sizeof(float) * kStages * kNC * ROW + 16 * kStages;
};

template <int K, int S, int OMAX, bool kInt>
__global__ void __launch_bounds__(kThreads, 1) dedisperse_kernel(DedispArgs a) {
  using Sh = Shape<K, S, OMAX>;
  constexpr int TT = Sh::TT, L = Sh::L, ROW = Sh::ROW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* srow = reinterpret_cast<float*>(smem_raw);                                    // [kStages][kNC][ROW]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(float) * kStages * kNC * ROW);

  const int tile = blockIdx.x % a.ntiles;
  const int tt = blockIdx.x / a.ntiles;
  const DmTile dt = a.tiles[tile];
  const int64_t t0 = (int64_t)tt * TT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchan = a.nchan;
  const int32_t* __restrict__ delay = a.delay;
  const int d_last = dt.d0 + dt.nd - 1;
  const int dw0 = dt.d0 + warp * K;             // first DM of this warp's group
  const bool warp_live = warp * K < dt.nd;
  const int nstage = (nchan + kNC - 1) / kNC;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Producer: stage i copies channels [i kNC, i kNC + kNC) into buffer i % kStages.
  auto produce = [&](int i) {
    const int buf = i % kStages;
    const int cb = i * kNC;
    unsigned total = 0;
    unsigned bytes[kNC];
    const float* src[kNC];
#pragma unroll
    for (int ci = 0; ci < kNC; ++ci) {
      const int c = cb + ci;
      bytes[ci] = 0;
      src[ci] = nullptr;
      if (c < nchan) {
        const int lo = delay[(int64_t)dt.d0 * nchan + c];
        const int hi = delay[(int64_t)d_last * nchan + c];
        const int64_t base = (t0 + lo) & ~int64_t(3);
        const int64_t end = t0 + TT + hi + 4;
        const int64_t n = ((end - base) + 3) & ~int64_t(3);
        bytes[ci] = (unsigned)(n * 4);
        src[ci] = a.y + (int64_t)c * a.ypitch + base;
        total += bytes[ci];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bars[buf], total);
#pragma unroll
    for (int ci = 0; ci < kNC; ++ci)
      if (bytes[ci]) bulk_g2s(srow + (buf * kNC + ci) * ROW, src[ci], bytes[ci], &bars[buf]);
  };

  if (threadIdx.x == 0)
    for (int i = 0; i < kStages && i < nstage; ++i) produce(i);

  float acc[K][S];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[j][s] = 0.f;

  bool failed = false;
  for (int i = 0; i < nstage; ++i) {
    const int buf = i % kStages;
    const int cb = i * kNC;
    // delays of this stage's channels for the warp's DMs (issued before the wait)
    int dv = 0;
    {
      const int ci = lane / (K + 1), j = lane % (K + 1);
      const int c = cb + ci;
      if (ci < kNC && c < nchan) {
        const int d = j < K ? (dw0 + j <= d_last ? dw0 + j : d_last) : dt.d0;
        dv = delay[(int64_t)d * nchan + c];
      }
    }
    bool ready = false;
    for (long long spin = 0; spin < kSpinLimit; ++spin)
      if (mbar_try_wait(&bars[buf], (unsigned)((i / kStages) & 1))) {
        ready = true;
        break;
      }
    const int nc = nchan - cb < kNC ? nchan - cb : kNC;
    if (ready && warp_live) {
      for (int ci = 0; ci < nc; ++ci) {
        const int lo = __shfl_sync(0xffffffffu, dv, ci * (K + 1) + K);
        const int dw = __shfl_sync(0xffffffffu, dv, ci * (K + 1));
        const int64_t base = (t0 + lo) & ~int64_t(3);
        const int aw = (int)(t0 + dw - base);
        int o[K];
        int omax = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          o[j] = (aw & 3) + __shfl_sync(0xffffffffu, dv, ci * (K + 1) + j) - dw;
          omax = o[j] > omax ? o[j] : omax;
        }
        const float* r = srow + (buf * kNC + ci) * ROW + lane * S + (aw & ~3);
        const int nq = (S + omax + 3) >> 2;
        float w[L];
#pragma unroll
        for (int q = 0; q < L / 4; ++q) {
          if (q < nq) {
            const float4 v = *reinterpret_cast<const float4*>(r + 4 * q);
            w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
          } else {
            w[4 * q] = w[4 * q + 1] = w[4 * q + 2] = w[4 * q + 3] = 0.f;
          }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) add_shifted<S, L, OMAX>(o[j], acc[j], w);
      }
    }
    failed = __syncthreads_or(!ready) != 0;
    if (failed) {
      // let the copies already issued land (bounded) before the CTA exits
      if (threadIdx.x == 0) {
        for (int k = i + 1; k < nstage && k < i + kStages; ++k)
          for (long long spin = 0; spin < kSpinLimit; ++spin)
            if (mbar_try_wait(&bars[k % kStages], (unsigned)((k / kStages) & 1))) break;
        atomicExch(a.status, TP_ETIMEOUT);
      }
      return;
    }
    if (threadIdx.x == 0 && i + kStages < nstage) produce(i + kStages);
  }

  // epilogue
  if (!warp_live) return;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int d = dw0 + j;
    if (d > d_last) break;
    const int64_t tl = t0 + (int64_t)lane * S;
    if constexpr (kInt) {
      int* Drow = static_cast<int*>(a.D) + (int64_t)d * a.dpitch;
      long long s1 = 0, s2 = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int v = __float2int_rn(acc[j][s]);
        if (tl + s < a.nout) {
          Drow[tl + s] = v;
          s1 += v;
          s2 += (long long)v * v;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (lane == 0) static_cast<longlong2*>(a.row_part)[(int64_t)d * a.ntt + tt] = make_longlong2(s1, s2);
    } else {
      float* Drow = static_cast<float*>(a.D) + (int64_t)d * a.dpitch;
      float s1 = 0.f, s2 = 0.f;
      if (tl + S <= a.nout) {
#pragma unroll
        for (int s = 0; s < S; s += 4)
          *reinterpret_cast<float4*>(Drow + tl + s) =
              make_float4(acc[j][s], acc[j][s + 1], acc[j][s + 2], acc[j][s + 3]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          s1 += acc[j][s];
          s2 += acc[j][s] * acc[j][s];
        }
      } else {
#pragma unroll
        for (int s = 0; s < S; ++s)
          if (tl + s < a.nout) {
            Drow[tl + s] = acc[j][s];
            s1 += acc[j][s];
            s2 += acc[j][s] * acc[j][s];
          }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (lane == 0)
        static_cast<double2*>(a.row_part)[(int64_t)d * a.ntt + tt] = make_double2((double)s1, (double)s2);
    }
  }
}

template <int K, int S, int OMAX>
cudaError_t launch_shape(const DedispArgs& a, cudaStream_t s) {
  using Sh = Shape<K, S, OMAX>;
  const long long grid = (long long)a.ntiles * a.ntt;
  if (grid <= 0 || grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e;
  if (a.dtype == TP_U8) {
    e = cudaFuncSetAttribute(dedisperse_kernel<K, S, OMAX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Sh::smem);
    if (e != cudaSuccess) return e;
    dedisperse_kernel<K, S, OMAX, true><<<(unsigned)grid, kThreads, Sh::smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(dedisperse_kernel<K, S, OMAX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Sh::smem);
    if (e != cudaSuccess) return e;
    dedisperse_kernel<K, S, OMAX, false><<<(unsigned)grid, kThreads, Sh::smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

// Kernel shapes: (DMs per warp K, outputs per lane S, max in-window offset).
const KernelShape kShapes[kNumShapes] = {
    {4, 20, 36},  // adjacent DMs within 33 samples of each other
    {2, 28, 36},
    {1, 28, 4},
};

int shape_tile_t(int shape) { return 32 * kShapes[shape].S; }

cudaError_t launch_dedisperse(const DedispArgs& a, cudaStream_t s) {
  switch (a.shape) {
    case 0: return launch_shape<4, 20, 36>(a, s);
    case 1: return launch_shape<2, 28, 36>(a, s);
    default: return launch_shape<1, 28, 4>(a, s);
  }
}

}  // namespace tp
