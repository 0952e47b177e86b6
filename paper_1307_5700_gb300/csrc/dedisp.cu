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
#include <type_traits>

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

// acc0 += low half, acc1 += high half of a packed pair of 16-bit samples
// (kind 0: binary16, 1: bfloat16), FP32 accumulation.
template <int KIND>
__device__ __forceinline__ void add_pair_h(float& acc0, float& acc1, unsigned pr) {
  if constexpr (KIND == 0)
    asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n add.rn.f32.f16 %0, l, %0;\n add.rn.f32.f16 %1, h, %1;\n}"
        : "+f"(acc0), "+f"(acc1)
        : "r"(pr));
  else
    asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n add.rn.f32.bf16 %0, l, %0;\n add.rn.f32.bf16 %1, h, %1;\n}"
        : "+f"(acc0), "+f"(acc1)
        : "r"(pr));
}

// Staged sample formats.
constexpr int kModeF32 = 0;   // FP32 y (float data)
constexpr int kModeF16 = 1;   // binary16 x~ (binary16 data, and 8-bit data widened exactly)
constexpr int kModeBF16 = 2;  // bfloat16 x~

template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO>
struct Shape {
  static constexpr int EB = MODE == kModeF32 ? 4 : 2;                         // bytes per sample
  static constexpr int QS = 16 / EB;                                          // samples per 16 B
  static constexpr int TT = 32 * S;                                           // outputs per tile
  static constexpr int L = (S + OMAX + 1 + QS - 1) / QS * QS;                 // window samples
  static constexpr int LR = L * EB / 4;                                       // window registers
  static constexpr int ROW = (TT + kMaxOverhang + OMAX + 2 * QS + 63) / 64 * 64;  // staged samples
  static constexpr int ROWB = ROW * EB;
  static constexpr int THREADS = (NCONS + 1) * 32;                            // + one producer warp
  static constexpr size_t data_bytes = (size_t)kStages * kNC * ROWB;
  static constexpr size_t del_bytes = sizeof(int) * kStages * kNC * 32;
  static constexpr size_t info_bytes = sizeof(int4) * kStages * kNC * NCONS;
  static constexpr size_t smem = data_bytes + del_bytes + info_bytes + 16 * kStages;
  // no bank conflicts: register windows (ALGO 0) start an odd number of 16-byte
  // units apart, direct 32-bit loads (ALGO 1) an odd number of words apart
  static_assert(ALGO == 1 ? ((S * EB / 4) % 2 == 1) : ((S * EB / 16) % 2 == 1), "lane stride");
  static_assert(ALGO == 0 || MODE == kModeF32 || S % 2 == 0, "16-bit direct loads pair samples");
};

// Per (stage, channel, consumer warp) the producer writes an int4:
//   x = byte offset of lane 0's window in shared memory,
//   y = byte j: in-window offset of DM j of the warp's group,
//   z = number of 16-byte units of the window the channel needs.

template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
__global__ void __launch_bounds__(Shape<K, S, OMAX, NCONS, MODE, ALGO>::THREADS, MINB)
    dedisperse_kernel(BatchArgs ba) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO>;
  // the CTA's beam: last b with cta_start[b] <= blockIdx.x
  int bi = 0;
  {
    int lo = 0, hi = ba.nbeams - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ba.cta_start[mid] <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    bi = lo;
  }
  const DedispArgs& a = ba.beams[bi];
  const int local = (int)blockIdx.x - ba.cta_start[bi];
  constexpr int TT = Sh::TT, LR = Sh::LR, ROWB = Sh::ROWB, EB = Sh::EB, QS = Sh::QS;
  static_assert(NCONS * K <= 32, "a producer lane holds one DM of the tile");
  static_assert(OMAX < 256, "offsets are packed in bytes");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* srow = smem_raw;                                                     // [kStages][kNC][ROWB]
  int* sdel = reinterpret_cast<int*>(smem_raw + Sh::data_bytes);                       // [kStages][kNC][32]
  int4* sinfo = reinterpret_cast<int4*>(smem_raw + Sh::data_bytes + Sh::del_bytes);      // [kStages][kNC][NCONS]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + Sh::data_bytes + Sh::del_bytes + Sh::info_bytes);
  uint64_t* empty = full + kStages;

  const int tile = local % a.ntiles;
  const int tt = local / a.ntiles;
  const DmTile dt = a.tiles[tile];
  const int64_t t0 = (int64_t)tt * TT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchan = a.nchan;
  const int nstage = (nchan + kNC - 1) / kNC;
  const int last = dt.nd - 1;
  const unsigned char* ybytes = static_cast<const unsigned char*>(a.y);

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
        const int64_t base = (t0 + lo) & ~int64_t(QS - 1);
        const int aw = (int)(t0 + dw - base);
        if constexpr (ALGO == 1) {
          // sample offset, in the staged row, of each DM's first output of lane 0
          int o[4] = {0, 0, 0, 0};
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const int jj = g0 + j <= last ? g0 + j : last;
            o[j] = (int)(t0 + del[ci * 32 + jj] - base);
          }
          sinfo[(buf * kNC + ci) * NCONS + w] =
              make_int4((buf * kNC + ci) * ROWB, o[0] | (o[1] << 16), o[2] | (o[3] << 16), 0);
          continue;
        }
        int offs = 0, omax = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int jj = g0 + j <= last ? g0 + j : last;
          int o = (aw & (QS - 1)) + del[ci * 32 + jj] - dw;
          // the planner bounds o by OMAX; the clamp keeps the indexed branch
          // inside its table whatever the delays hold
          o = o < 0 ? 0 : (o > OMAX ? OMAX : o);
          offs |= o << (8 * j);
          omax = o > omax ? o : omax;
        }
        sinfo[(buf * kNC + ci) * NCONS + w] =
            make_int4((buf * kNC + ci) * ROWB + (aw & ~(QS - 1)) * EB, offs, (S + omax + QS - 1) / QS, 0);
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
          const int64_t base = (t0 + lo) & ~int64_t(QS - 1);
          const int64_t end = t0 + TT + hi + QS;
          bytes[ci] = (unsigned)((((end - base) * EB) + 15) & ~int64_t(15));
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
          const int64_t base = (t0 + cur[ci]) & ~int64_t(QS - 1);
          bulk_g2s(srow + (buf * kNC + ci) * ROWB, ybytes + ((int64_t)c * a.ypitch + base) * EB, bytes[ci],
                   &full[buf]);
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
  using WT = typename std::conditional<MODE == kModeF32, float, unsigned>::type;
  WT w[ALGO == 0 ? LR : 4];
#pragma unroll
  for (int q = 0; q < (ALGO == 0 ? LR : 4); ++q) w[q] = 0;

  for (int i = 0; i < nstage; ++i) {
    const int buf = i % kStages;
    if (!mbar_wait_bounded(&full[buf], (unsigned)((i / kStages) & 1))) {
      if (lane == 0) atomicExch(a.status, TP_ETIMEOUT);
      return;
    }
    const int nc = nchan - i * kNC < kNC ? nchan - i * kNC : kNC;
    if (live && ALGO == 1) {
      // direct loads: each DM reads its own S samples at its own offset
      for (int ci = 0; ci < nc; ++ci) {
        const int4 inf = sinfo[(buf * kNC + ci) * NCONS + warp];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int oj = ((j < 2 ? inf.y : inf.z) >> (16 * (j & 1))) & 0xffff;
          const int p = oj + lane * S;
          if constexpr (MODE == kModeF32) {
            const float* r = reinterpret_cast<const float*>(srow + inf.x) + p;
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) acc[j][s2] += r[s2];
          } else {
            // words holding samples p .. p + S (two per word); an odd start
            // shifts every pair by one half-word
            const unsigned* r = reinterpret_cast<const unsigned*>(srow + inf.x) + (p >> 1);
            const unsigned sel = (p & 1) ? 0x5432u : 0x3210u;
            unsigned wv[S / 2 + 1];
#pragma unroll
            for (int k = 0; k <= S / 2; ++k) wv[k] = r[k];
#pragma unroll
            for (int k = 0; k < S / 2; ++k) {
              const unsigned pr = __byte_perm(wv[k], wv[k + 1], sel);
              add_pair_h<MODE == kModeBF16 ? 1 : 0>(acc[j][2 * k], acc[j][2 * k + 1], pr);
            }
          }
        }
      }
    } else if (live) {
      for (int ci = 0; ci < nc; ++ci) {
        const int4 inf = sinfo[(buf * kNC + ci) * NCONS + warp];
        const unsigned char* r = srow + inf.x + lane * S * EB;
#pragma unroll
        for (int q = 0; q < LR / 4; ++q) {
          if (q < inf.z) {
            if constexpr (MODE == kModeF32) {
              const float4 v = *reinterpret_cast<const float4*>(r + 16 * q);
              w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
            } else {
              const uint4 v = *reinterpret_cast<const uint4*>(r + 16 * q);
              w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int o = (inf.y >> (8 * j)) & 0xff;
          if constexpr (ALGO == 0) {
            if constexpr (MODE == kModeF32)
              add_shifted<S, LR, OMAX>(o, acc[j], w);
            else
              add_shifted_h<S, LR, OMAX, MODE == kModeBF16 ? 1 : 0>(o, acc[j], w);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[buf]);
  }

  // epilogue: 16-bit modes accumulated the stored samples x~; subtract the
  // block's sum of bandpass values (exact integers for 8-bit data)
  if (!live) return;
  const bool is_int = a.dtype == TP_U8;
  float bhi = 0.f, blo = 0.f;
  int bint = 0;
  if constexpr (MODE != kModeF32) {
    const double bs = *a.bsum;
    bhi = (float)bs;
    blo = (float)(bs - (double)bhi);
    bint = (int)bs;
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (g0 + j > last) break;
    const int d = dt.d0 + g0 + j;
    const int64_t tl = t0 + (int64_t)lane * S;
    if (is_int) {
      int* Drow = static_cast<int*>(a.D) + (int64_t)d * a.dpitch;
      long long s1 = 0, s2 = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int v = __float2int_rn(acc[j][s]) - bint;
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
      if constexpr (MODE != kModeF32) {
#pragma unroll
        for (int s = 0; s < S; ++s) acc[j][s] = (acc[j][s] - bhi) - blo;
      }
      float* Drow = static_cast<float*>(a.D) + (int64_t)d * a.dpitch;
      float s1 = 0.f, s2 = 0.f;
      if (S % 4 == 0 && tl + S <= a.nout) {
#pragma unroll
        for (int s = 0; s < (S / 4) * 4; s += 4)
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

template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
cudaError_t launch_mode(const BatchArgs& ba, int ctas, cudaStream_t s) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO>;
  if (ctas <= 0) return cudaErrorInvalidValue;
  auto k = dedisperse_kernel<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)ctas, Sh::THREADS, Sh::smem, s>>>(ba);
  return cudaGetLastError();
}

template <int K, int S, int OMAX, int NCONS, int EB, int ALGO, int MINB>
cudaError_t launch_shape(const BatchArgs& ba, int dtype, int ctas, cudaStream_t s) {
  if constexpr (EB == 4) {
    return launch_mode<K, S, OMAX, NCONS, kModeF32, ALGO, MINB>(ba, ctas, s);
  } else {
    if (dtype == TP_BF16) return launch_mode<K, S, OMAX, NCONS, kModeBF16, ALGO, MINB>(ba, ctas, s);
    return launch_mode<K, S, OMAX, NCONS, kModeF16, ALGO, MINB>(ba, ctas, s);
  }
}

}  // namespace

// Kernel shapes: (DMs per warp K, outputs per lane S, largest in-window offset
// OMAX, consumer warps).  The planner keeps the shapes whose K-trial groups
// all spread by at most OMAX - 3 samples; the autotuner (or the first
// feasible shape) picks among them.
// EB = bytes per staged sample: 4 for FP32 data, 2 for 16-bit and 8-bit data.
// ALGO 0: register window + jump-table shifted adds (reuse across the K DMs);
// ALGO 1: direct shared loads per DM (no offset bound, OMAX unused).
// MINB: CTAs per SM the register allocation is sized for.
#define TP_SHAPES(X)                 \
  X(0, 4, 20, 36, 8, 4, 0, 1)        \
  X(1, 2, 20, 16, 12, 4, 0, 1)       \
  X(2, 2, 28, 16, 8, 4, 0, 1)        \
  X(3, 3, 20, 24, 8, 4, 0, 1)        \
  X(4, 4, 12, 52, 8, 4, 0, 1)        \
  X(5, 2, 20, 24, 12, 4, 0, 1)       \
  X(6, 1, 28, 4, 16, 4, 0, 1)        \
  X(7, 4, 24, 40, 8, 2, 0, 1)        \
  X(8, 2, 24, 24, 12, 2, 0, 1)       \
  X(9, 4, 8, 60, 8, 2, 0, 1)         \
  X(10, 2, 24, 32, 12, 2, 0, 1)      \
  X(11, 1, 24, 8, 16, 2, 0, 1)       \
  X(12, 2, 27, 0, 8, 4, 1, 2)        \
  X(13, 4, 15, 0, 8, 4, 1, 2)        \
  X(14, 2, 26, 0, 8, 2, 1, 2)        \
  X(15, 4, 22, 0, 8, 2, 1, 1)        \
  X(16, 2, 22, 0, 16, 2, 1, 1)

#define TP_SHAPE_ENTRY(i, K, S, O, N, EB, A, M) {K, S, O, N, EB, A},
const KernelShape kShapes[kNumShapes] = {TP_SHAPES(TP_SHAPE_ENTRY)};
#undef TP_SHAPE_ENTRY

int shape_tile_t(int shape) { return 32 * kShapes[shape].S; }

cudaError_t launch_dedisperse(int shape, int dtype, const BatchArgs& ba, int ctas, cudaStream_t s) {
  switch (shape) {
#define TP_SHAPE_CASE(i, K, S, O, N, EB, A, M) \
  case i: return launch_shape<K, S, O, N, EB, A, M>(ba, dtype, ctas, s);
    TP_SHAPES(TP_SHAPE_CASE)
#undef TP_SHAPE_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tp
