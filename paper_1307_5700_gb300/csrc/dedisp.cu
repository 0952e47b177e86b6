// A5: brute-force incoherent dedispersion (Sec. 2.2.2, delays of Eq. 1)
//
//   D[d][t] = sum_{c=0}^{nchan-1} y[c][t + delay[d][c]],   0 <= t < T,
//
// over the substituted, bandpass-corrected series y written by the A3/A4
// kernel (FP32; exact small integers for 8-bit data).
//
// Work decomposition.  A CTA owns a tile of consecutive DM trials (up to 8
// groups of K) x TT = 32 S output samples.  Warps 0-7 are consumers: warp w
// owns group w, lane l owns the S consecutive outputs t0 + l S .. + S - 1 of
// each of the K DMs.  Warp 8 is the producer: for each pipeline stage (kNC
// channels) it stages the stage's delays for the tile's DMs into shared memory
// and copies, per channel, the samples the tile needs,
// [t0 + delay[d_first][c], t0 + TT + delay[d_last][c]) rounded out to 16 B,
// with cp.async.bulk onto a "full" mbarrier; consumers release a stage on an
// "empty" mbarrier (kStages stages in flight, no CTA-wide barrier).
// A consumer lane loads a register window of S + spread + 4 samples with
// 128-bit shared loads (only as many quads as this channel's spread needs) and
// adds it into the K x S accumulators at each DM's offset inside the window:
// the offsets are warp-uniform run-time values, so each DM jumps through a
// table (brx.idx) into one of OMAX + 1 unrolled add sequences
// (dispatch_gen.cuh).  Every sample loaded from shared memory thus feeds up to
// K adds from registers.  Each (d, t) adds its channels in index order (FP32).
// Every mbarrier wait is bounded; a wait that gives up records TP_ETIMEOUT in
// the beam's status word and the CTA leaves after letting its copies land.
//
// The epilogue writes D (FP32, or int32 for 8-bit data, exact) and per
// (DM, time tile) sums of D and D^2 for the series statistics of A6.
#include <cstdint>

#include "dispatch_gen.cuh"
#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kNC = 4;                              // channels per pipeline stage
constexpr int kStages = 4;                          // pipeline depth
constexpr long long kSpinLimit = 1LL << 24;         // bounded mbarrier waits

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (long long spin = 0; spin < kSpinLimit; ++spin)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <int K, int S, int OMAX, int NCONS>
struct Shape {
  static constexpr int TT = 32 * S;                                          // outputs per tile
  static constexpr int L = (S + OMAX + 1 + 3) / 4 * 4;                       // register window
  static constexpr int ROW = (TT + kMaxOverhang + OMAX + 8 + 31) / 32 * 32;  // staged floats per channel
  static constexpr int THREADS = (NCONS + 1) * 32;                           // + one producer warp
  static constexpr size_t data_bytes = sizeof(float) * kStages * kNC * ROW;
  static constexpr size_t del_bytes = sizeof(int) * kStages * kNC * 32;
  static constexpr size_t info_bytes = sizeof(int4) * kStages * kNC * NCONS;
  static constexpr size_t smem = data_bytes + del_bytes + info_bytes + 16 * kStages;
};

// Per (stage, channel, consumer warp): where the warp's window starts in
// shared memory, the K in-window offsets (one byte each) and how many quads
// of the window the channel needs.  Written by the producer.
struct WarpChan {
  int roff;    // float offset of lane 0's window
  int offs;    // byte j = offset of DM j of the warp's group
  int nq;      // window quads to load
  int pad;
};

template <int K, int S, int OMAX, int NCONS, bool kInt>
__global__ void __launch_bounds__(Shape<K, S, OMAX, NCONS>::THREADS, 1) dedisperse_kernel(DedispArgs a) {
  using Sh = Shape<K, S, OMAX, NCONS>;
  constexpr int TT = Sh::TT, L = Sh::L, ROW = Sh::ROW;
  static_assert(NCONS * K <= 32, "a producer lane holds one DM of the tile");
  static_assert(OMAX < 256, "offsets are packed in bytes");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* srow = reinterpret_cast<float*>(smem_raw);                               // [kStages][kNC][ROW]
  int* sdel = reinterpret_cast<int*>(smem_raw + Sh::data_bytes);                   // [kStages][kNC][32]
  int4* sinfo = reinterpret_cast<int4*>(smem_raw + Sh::data_bytes + Sh::del_bytes);  // [kStages][kNC][NCONS]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + Sh::data_bytes + Sh::del_bytes + Sh::info_bytes);
  uint64_t* empty = full + kStages;

  const int tile = blockIdx.x % a.ntiles;
  const int tt = blockIdx.x / a.ntiles;
  const DmTile dt = a.tiles[tile];
  const int64_t t0 = (int64_t)tt * TT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchan = a.nchan;
  const int nstage = (nchan + kNC - 1) / kNC;
  const int last = dt.nd - 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NCONS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NCONS) {
    // ---------------------------------------------------------------- producer
    // lane j < nd holds delayT[c][d0 + j] for the kNC channels of a stage
    const int32_t* __restrict__ dT = a.delayT;
    auto fetch = [&](int i, int (&v)[kNC]) {
#pragma unroll
      for (int ci = 0; ci < kNC; ++ci) {
        const int c = i * kNC + ci;
        v[ci] = (c < nchan && lane < dt.nd) ? __ldg(dT + (int64_t)c * a.dtpitch + dt.d0 + lane) : 0;
      }
    };
    int cur[kNC], nxt[kNC];
    if (nstage > 0) fetch(0, cur);
    bool ok = true;
    int issued = 0;
    for (int i = 0; i < nstage; ++i) {
      if (i + 1 < nstage) fetch(i + 1, nxt);
      const int buf = i % kStages;
      if (i >= kStages) {
        bool got = false;
        if (lane == 0) got = mbar_wait_bounded(&empty[buf], (unsigned)(((i / kStages) - 1) & 1));
        if (!__shfl_sync(0xffffffffu, got, 0)) {
          ok = false;
          break;
        }
      }
      int* del = sdel + buf * kNC * 32;
#pragma unroll
      for (int ci = 0; ci < kNC; ++ci) del[ci * 32 + lane] = cur[ci];
      __syncwarp();
      // window geometry of every (channel, consumer warp) pair of the stage
      for (int p = lane; p < kNC * NCONS; p += 32) {
        const int ci = p / NCONS, w = p % NCONS;
        const int g0 = w * K < last ? w * K : last;
        const int lo = del[ci * 32];
        const int dw = del[ci * 32 + g0];
        const int64_t base = (t0 + lo) & ~int64_t(3);
        const int aw = (int)(t0 + dw - base);
        int offs = 0, omax = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int jj = g0 + j <= last ? g0 + j : last;
          int o = (aw & 3) + del[ci * 32 + jj] - dw;
          // the planner bounds o by OMAX; the clamp keeps the indexed branch
          // inside its table whatever the delays hold
          o = o < 0 ? 0 : (o > OMAX ? OMAX : o);
          offs |= o << (8 * j);
          omax = o > omax ? o : omax;
        }
        sinfo[(buf * kNC + ci) * NCONS + w] =
            make_int4((buf * kNC + ci) * ROW + (aw & ~3), offs, (S + omax + 3) >> 2, 0);
      }
      unsigned bytes[kNC];
      unsigned total = 0;
#pragma unroll
      for (int ci = 0; ci < kNC; ++ci) {
        const int lo = __shfl_sync(0xffffffffu, cur[ci], 0);
        const int hi = __shfl_sync(0xffffffffu, cur[ci], last);
        const int c = i * kNC + ci;
        bytes[ci] = 0;
        if (c < nchan) {
          const int64_t base = (t0 + lo) & ~int64_t(3);
          const int64_t end = t0 + TT + hi + 4;
          bytes[ci] = (unsigned)((((end - base) + 3) & ~int64_t(3)) * 4);
          total += bytes[ci];
        }
      }
      __syncwarp();
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&full[buf], total);
#pragma unroll
        for (int ci = 0; ci < kNC; ++ci) {
          if (!bytes[ci]) continue;
          const int c = i * kNC + ci;
          const int64_t base = (t0 + cur[ci]) & ~int64_t(3);
          bulk_g2s(srow + (buf * kNC + ci) * ROW, a.y + (int64_t)c * a.ypitch + base, bytes[ci], &full[buf]);
        }
      }
      ++issued;
#pragma unroll
      for (int ci = 0; ci < kNC; ++ci) cur[ci] = nxt[ci];
    }
    // let every issued copy land before the CTA can exit
    if (lane == 0) {
      for (int k = issued - 1; k >= 0 && k >= issued - kStages; --k)
        if (!mbar_wait_bounded(&full[k % kStages], (unsigned)((k / kStages) & 1))) ok = false;
      if (!ok) atomicExch(a.status, TP_ETIMEOUT);
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const int g0 = warp * K;                 // first tile-local DM of this warp
  const bool live = g0 < dt.nd;

  float acc[K][S];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[j][s] = 0.f;
  float w[L];
#pragma unroll
  for (int q = 0; q < L; ++q) w[q] = 0.f;

  for (int i = 0; i < nstage; ++i) {
    const int buf = i % kStages;
    if (!mbar_wait_bounded(&full[buf], (unsigned)((i / kStages) & 1))) {
      if (lane == 0) atomicExch(a.status, TP_ETIMEOUT);
      return;
    }
    const int nc = nchan - i * kNC < kNC ? nchan - i * kNC : kNC;
    if (live) {
      for (int ci = 0; ci < nc; ++ci) {
        const int4 inf = sinfo[(buf * kNC + ci) * NCONS + warp];
        const float* r = srow + inf.x + lane * S;
#pragma unroll
        for (int q = 0; q < L / 4; ++q) {
          if (q < inf.z) {
            const float4 v = *reinterpret_cast<const float4*>(r + 4 * q);
            w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
          }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) add_shifted<S, L, OMAX>((inf.y >> (8 * j)) & 0xff, acc[j], w);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[buf]);
  }

  // epilogue
  if (!live) return;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (g0 + j > last) break;
    const int d = dt.d0 + g0 + j;
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

template <int K, int S, int OMAX, int NCONS>
cudaError_t launch_shape(const DedispArgs& a, cudaStream_t s) {
  using Sh = Shape<K, S, OMAX, NCONS>;
  const long long grid = (long long)a.ntiles * a.ntt;
  if (grid <= 0 || grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e;
  if (a.dtype == TP_U8) {
    auto k = dedisperse_kernel<K, S, OMAX, NCONS, true>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, Sh::THREADS, Sh::smem, s>>>(a);
  } else {
    auto k = dedisperse_kernel<K, S, OMAX, NCONS, false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)grid, Sh::THREADS, Sh::smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

// Kernel shapes: (DMs per warp K, outputs per lane S, largest in-window offset
// OMAX, consumer warps).  The planner keeps the shapes whose K-trial groups
// all spread by at most OMAX - 3 samples; the autotuner (or the first
// feasible shape) picks among them.
#define TP_SHAPES(X)      \
  X(0, 4, 20, 36, 8)      \
  X(1, 2, 20, 16, 12)     \
  X(2, 2, 28, 16, 8)      \
  X(3, 3, 20, 24, 8)      \
  X(4, 4, 12, 52, 8)      \
  X(5, 2, 20, 24, 12)     \
  X(6, 1, 28, 4, 16)

#define TP_SHAPE_ENTRY(i, K, S, O, N) {K, S, O, N},
const KernelShape kShapes[kNumShapes] = {TP_SHAPES(TP_SHAPE_ENTRY)};
#undef TP_SHAPE_ENTRY

int shape_tile_t(int shape) { return 32 * kShapes[shape].S; }

cudaError_t launch_dedisperse(const DedispArgs& a, cudaStream_t s) {
  switch (a.shape) {
#define TP_SHAPE_CASE(i, K, S, O, N) \
  case i: return launch_shape<K, S, O, N>(a, s);
    TP_SHAPES(TP_SHAPE_CASE)
#undef TP_SHAPE_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tp
