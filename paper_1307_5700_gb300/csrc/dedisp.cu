// A4-A5: substitution of flagged samples and brute-force incoherent
// dedispersion (Sec. 2.2.2, delays of Eq. 1):
//
//   D[d][t] = sum_{c=0}^{nchan-1} y[c][t + delay[d][c]],   0 <= t < T,
//   y[c][u] = 0 where (c, u) is flagged, else x[c][u] - b_c.
//
// One CTA owns a tile of up to 32 consecutive DM trials x 512 output samples.
// It walks the channels in order, 8 at a time: the samples a channel
// contributes to the tile, [t0 + delay[d_first][c], t0 + 512 + delay[d_last][c]),
// are staged once into shared memory with the bandpass subtracted and the
// flags applied (y is never written to HBM), and then every DM of the tile reads
// its shifted 512-sample window from that copy.  Each (d, t) accumulates its
// channels in index order: in FP32 for float data (binary16 / bfloat16 are
// widened exactly), in int32 for 8-bit data (exact).
//
// Warp w holds DMs w, w + 8, w + 16, w + 24 of the tile; lane l holds samples
// t0 + l + 32 s, s < 16, so every shared-memory read of a warp is 32
// consecutive words (conflict-free) and every store of D is a coalesced
// 128-byte line.  The epilogue writes D and per-(DM, time-tile) sums of D and
// D^2 for the series statistics of A6.
#include <cstdint>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kCB = 8;                          // channels per stage
constexpr int kSlot = kTileT + kMaxOverhang;    // staged samples per channel
constexpr int kPerLane = kTileT / 32;           // outputs per lane per DM
constexpr int kDmPerWarp = kMaxTileDm / 8;

template <int DT>
__device__ __forceinline__ float load_f(const void* x, int64_t i);
template <>
__device__ __forceinline__ float load_f<TP_F32>(const void* x, int64_t i) {
  return __ldg(static_cast<const float*>(x) + i);
}
template <>
__device__ __forceinline__ float load_f<TP_F16>(const void* x, int64_t i) {
  unsigned short h = __ldg(static_cast<const unsigned short*>(x) + i);
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
  return f;
}
template <>
__device__ __forceinline__ float load_f<TP_BF16>(const void* x, int64_t i) {
  unsigned short h = __ldg(static_cast<const unsigned short*>(x) + i);
  return __uint_as_float((unsigned)h << 16);
}

template <int DT>
struct Acc {
  using T = float;
};
template <>
struct Acc<TP_U8> {
  using T = int;
};

template <int DT>
__device__ __forceinline__ typename Acc<DT>::T corrected(const DedispArgs& a, int c, int64_t g,
                                                         bool check, float mh, float ml, int b) {
  bool f = false;
  if (check) {
    const bool chunk = a.chan_nflag[c] != 0 && a.chunk_flag[(int64_t)c * a.nchunk + g / a.W];
    const bool spec = (a.spec_bits[g >> 5] >> (g & 31)) & 1u;
    f = chunk || spec;
  }
  if constexpr (DT == TP_U8) {
    const int v = __ldg(static_cast<const unsigned char*>(a.x) + (int64_t)c * a.pitch + g);
    return f ? 0 : v - b;
  } else {
    const float v = load_f<DT>(a.x, (int64_t)c * a.pitch + g);
    return f ? 0.f : (v - mh) - ml;
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads, 2) dedisperse_kernel(DedispArgs a) {
  using AT = typename Acc<DT>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AT* sy = reinterpret_cast<AT*>(smem_raw);                   // [2][kCB][kSlot]
  int* soff = reinterpret_cast<int*>(sy + 2 * kCB * kSlot);   // [2][kCB][kMaxTileDm]

  const int tile = blockIdx.x % a.ntiles;
  const int tt = blockIdx.x / a.ntiles;
  const DmTile dt = a.tiles[tile];
  const int64_t t0 = (int64_t)tt * kTileT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool any_spec = *a.spec_nflag != 0;

  AT acc[kDmPerWarp][kPerLane];
#pragma unroll
  for (int i = 0; i < kDmPerWarp; ++i)
#pragma unroll
    for (int s = 0; s < kPerLane; ++s) acc[i][s] = 0;

  auto stage = [&](int cbase, int buf) {
    AT* dst = sy + buf * kCB * kSlot;
    int* off = soff + buf * kCB * kMaxTileDm;
    for (int i = threadIdx.x; i < kCB * kMaxTileDm; i += kThreads) {
      const int ci = i / kMaxTileDm, j = i % kMaxTileDm;
      const int c = cbase + ci;
      int v = 0;
      if (c < a.nchan && j < dt.nd)
        v = a.delay[(int64_t)(dt.d0 + j) * a.nchan + c] - a.delay[(int64_t)dt.d0 * a.nchan + c];
      off[i] = v;
    }
    for (int ci = 0; ci < kCB; ++ci) {
      const int c = cbase + ci;
      if (c >= a.nchan) break;
      const int lo = a.delay[(int64_t)dt.d0 * a.nchan + c];
      const int hi = a.delay[(int64_t)(dt.d0 + dt.nd - 1) * a.nchan + c];
      const int span = kTileT + hi - lo;
      const int64_t base = t0 + lo;
      const bool check = any_spec || a.chan_nflag[c] != 0;
      float mh = 0.f, ml = 0.f;
      int b = 0;
      if constexpr (DT == TP_U8) {
        b = a.bint[c];
      } else {
        mh = a.mu_hi[c];
        ml = a.mu_lo[c];
      }
      AT* row = dst + ci * kSlot;
      for (int u = threadIdx.x; u < span; u += kThreads) {
        const int64_t g = base + u;
        row[u] = g < a.nsamp ? corrected<DT>(a, c, g, check, mh, ml, b) : AT(0);
      }
    }
  };

  stage(0, 0);
  __syncthreads();
  int buf = 0;
  for (int cb = 0; cb < a.nchan; cb += kCB, buf ^= 1) {
    if (cb + kCB < a.nchan) stage(cb + kCB, buf ^ 1);
    const AT* src = sy + buf * kCB * kSlot;
    const int* off = soff + buf * kCB * kMaxTileDm;
    const int nc = a.nchan - cb < kCB ? a.nchan - cb : kCB;
    for (int ci = 0; ci < nc; ++ci) {
#pragma unroll
      for (int i = 0; i < kDmPerWarp; ++i) {
        const int slot = warp + 8 * i;
        if (slot < dt.nd) {
          const AT* r = src + ci * kSlot + off[ci * kMaxTileDm + slot] + lane;
#pragma unroll
          for (int s = 0; s < kPerLane; ++s) acc[i][s] += r[32 * s];
        }
      }
    }
    __syncthreads();
  }

  // epilogue: D and per-tile row sums
#pragma unroll
  for (int i = 0; i < kDmPerWarp; ++i) {
    const int slot = warp + 8 * i;
    if (slot >= dt.nd) continue;
    const int d = dt.d0 + slot;
    AT* Drow = static_cast<AT*>(a.D) + (int64_t)d * a.dpitch;
    if constexpr (DT == TP_U8) {
      long long s1 = 0, s2 = 0;
#pragma unroll
      for (int s = 0; s < kPerLane; ++s) {
        const int64_t t = t0 + lane + 32 * s;
        if (t < a.nout) {
          Drow[t] = acc[i][s];
          s1 += acc[i][s];
          s2 += (long long)acc[i][s] * acc[i][s];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      }
      if (lane == 0)
        static_cast<longlong2*>(a.row_part)[(int64_t)d * a.ntt + tt] = make_longlong2(s1, s2);
    } else {
      float s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int s = 0; s < kPerLane; ++s) {
        const int64_t t = t0 + lane + 32 * s;
        if (t < a.nout) {
          Drow[t] = acc[i][s];
          s1 += acc[i][s];
          s2 += acc[i][s] * acc[i][s];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      }
      if (lane == 0)
        static_cast<double2*>(a.row_part)[(int64_t)d * a.ntt + tt] =
            make_double2((double)s1, (double)s2);
    }
  }
}

template <int DT>
cudaError_t launch_t(const DedispArgs& a, cudaStream_t s) {
  using AT = typename Acc<DT>::T;
  const size_t smem = sizeof(AT) * 2 * kCB * kSlot + sizeof(int) * 2 * kCB * kMaxTileDm;
  cudaError_t e = cudaFuncSetAttribute(dedisperse_kernel<DT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = (long long)a.ntiles * a.ntt;
  if (grid <= 0 || grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  dedisperse_kernel<DT><<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dedisperse(const DedispArgs& a, cudaStream_t s) {
  switch (a.dtype) {
    case TP_U8: return launch_t<TP_U8>(a, s);
    case TP_F16: return launch_t<TP_F16>(a, s);
    case TP_BF16: return launch_t<TP_BF16>(a, s);
    default: return launch_t<TP_F32>(a, s);
  }
}

}  // namespace tp
