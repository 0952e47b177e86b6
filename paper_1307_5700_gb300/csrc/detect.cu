// A6-A7: per-DM series statistics (normalisation of Sec. 2.2.3) and the
// n-sigma detection of Sec. 2.3, compacted on the device.
//
//   mu_d = sum_t D / T,  sigma_d^2 = sum_t D^2 / T - mu_d^2   (population)
//   candidate (d, t)  <=>  sigma_d > 0  and  D[d][t] - mu_d >= nsigma * sigma_d
//
// row_stats (one CTA per DM) folds the per-(DM, time-tile) partial sums of the
// dedispersion epilogue (exact int64 for 8-bit data) into mu_d, sigma_d and
// turns the binary64 predicate into an equivalent threshold on the stored
// value: the predicate is monotone in D, so "D >= smallest passing value" is
// the same test, made once per row instead of once per sample.
// Compaction is deterministic and ordered by (d, t) without a sort:
//   count : one CTA per (d, 4096 samples) writes one hit bit per sample and
//           its hit count;
//   scan  : one CTA turns the counts into offsets (row-major in (d, block));
//   write : each CTA ranks its hits in t order (ballots + a 128-entry scan) and
//           writes records at offset + rank, keeping those below the capacity.
//
// Optional post-processing of Sec. 2.2.3 (median filter of Eq. 2, detrending
// and normalisation).  post_kernel (one CTA per (d, 4096 samples)) replaces
// each value by the median of the w values centred on it -- the series ends
// repeat -- selected with min/max exchanges (an exact selection of a stored
// value), writes the filtered series M, and sums per tile y, (t - t_c) y and
// y^2 (FP32 over a thread's 16 values, FP64 above; exact int64 for 8-bit
// data).  With detrending, row_stats fits the least-squares line
// y ~ mean + beta u_t, u_t = 2t - (T - 1), from those sums,
//   mean = Sy / T, beta = Suy / Suu, Suu = (T-1) T (T+1) / 3,
//   RSS = Syy - Sy Sy / T - Suy Suy / Suu, sigma = sqrt(max(RSS, 0) / T),
// and a sample is a candidate when y - (mean + beta u_t) >= nsigma sigma,
// evaluated in binary64 in that order whenever an FP32 pre-test cannot
// decide it with a wide margin.
#include <cfloat>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPer = kDetectT / kThreads;  // 16 samples per thread

__device__ __forceinline__ bool passes(double v, double mu, double thr) { return __dsub_rn(v, mu) >= thr; }

// The smallest int i with passes(i) (INT_MAX when none does): the predicate
// is monotone in i, so a bisection of the int range finds it in at most 32
// steps whatever the statistics hold.
__device__ __forceinline__ int smallest_passing_int(double mu, double thr) {
  long long lo = INT_MIN, hi = INT_MAX;
  if (!passes((double)hi, mu, thr)) return INT_MAX;
  while (lo < hi) {
    const long long mid = lo + (hi - lo) / 2;
    if (passes((double)mid, mu, thr)) hi = mid;
    else lo = mid + 1;
  }
  return (int)lo;
}

// detrended residual y - (mean + beta u), binary64 in the order written
__device__ __forceinline__ double residual(double v, double mean, double beta, double u) {
  return __dsub_rn(v, __dadd_rn(mean, __dmul_rn(beta, u)));
}

// compare-exchange: lo = min, hi = max (exact selections)
__device__ __forceinline__ void cx(float& lo, float& hi) {
  const float a = fminf(lo, hi), b = fmaxf(lo, hi);
  lo = a, hi = b;
}
__device__ __forceinline__ void cx(int& lo, int& hi) {
  const int a = min(lo, hi), b = max(lo, hi);
  lo = a, hi = b;
}

// median of v[0 .. W) (W odd): odd-even transposition sort, middle element
template <int W, typename V>
__device__ __forceinline__ V median_of(V (&v)[W]) {
#pragma unroll
  for (int pass = 0; pass < W; ++pass)
#pragma unroll
    for (int i = pass & 1; i + 1 < W; i += 2) cx(v[i], v[i + 1]);
  return v[W / 2];
}

constexpr int kPostHalo = kMaxMedianWidth / 2;

// Post-processing of one (d, 4096-sample tile): median filter (W > 1) and the
// tile's sums {y, (t - t_c) y, y^2}, t_c = tile start + 2048.
template <bool INT, int W>
__global__ void __launch_bounds__(kThreads) post_kernel(DetectArgs a) {
  using V = typename std::conditional<INT, int, float>::type;
  const int d = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * kDetectT;
  const int64_t T = a.nout;
  const V* row = static_cast<const V*>(a.D) + (int64_t)d * a.dpitch;
  constexpr int H = W / 2;
  __shared__ V s_v[kDetectT + 2 * kPostHalo];
  if constexpr (W > 1) {
    // s_v[i] = value at t0 - H + i, positions beyond the series taking the
    // end value: 16-byte loads for the tile, clamped loads for the halos
    using V4 = typename std::conditional<INT, int4, float4>::type;
    for (int q = threadIdx.x; q < kDetectT / 4; q += kThreads) {
      const int64_t t = t0 + 4 * q;
      if (t + 3 < T) {
        const V4 v = *reinterpret_cast<const V4*>(row + t);
        s_v[H + 4 * q] = v.x, s_v[H + 4 * q + 1] = v.y, s_v[H + 4 * q + 2] = v.z, s_v[H + 4 * q + 3] = v.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) s_v[H + 4 * q + e] = row[t + e < T ? t + e : T - 1];
      }
    }
    if (threadIdx.x < 2 * H) {
      const int i = threadIdx.x < H ? threadIdx.x : kDetectT + threadIdx.x;
      int64_t t = t0 - H + i;
      t = t < 0 ? 0 : (t > T - 1 ? T - 1 : t);
      s_v[i] = row[t];
    }
    __syncthreads();
  }
  V* mrow = static_cast<V*>(a.M) + (int64_t)d * a.dpitch;
  const int64_t tc = t0 + kDetectT / 2;
  float fs = 0.f, fd = 0.f, fq = 0.f;
  long long is = 0, id = 0, iq = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t tb = t0 + 1024 * r + 4 * threadIdx.x;
    V y[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if constexpr (W > 1) {
        V w[W];
        const int j = (int)(tb + e - t0);
#pragma unroll
        for (int k = 0; k < W; ++k) w[k] = s_v[j + k];
        y[e] = median_of<W>(w);
      } else {
        y[e] = tb + e < T ? row[tb + e] : V(0);
      }
    }
    if constexpr (W > 1) {
      if (tb + 3 < T) {
        if constexpr (INT)
          *reinterpret_cast<int4*>(mrow + tb) = make_int4(y[0], y[1], y[2], y[3]);
        else
          *reinterpret_cast<float4*>(mrow + tb) = make_float4(y[0], y[1], y[2], y[3]);
      } else {
        for (int e = 0; e < 4; ++e)
          if (tb + e < T) mrow[tb + e] = y[e];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (tb + e >= T) continue;
      const int dt = (int)(tb + e - tc);
      if constexpr (INT) {
        is += y[e];
        id += (long long)dt * y[e];
        iq += (long long)y[e] * y[e];
      } else {
        fs += y[e];
        fd += (float)dt * y[e];
        fq += y[e] * y[e];
      }
    }
  }
  __shared__ double s_f[3][kWarps];
  __shared__ long long s_i[3][kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (INT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      is += __shfl_xor_sync(0xffffffffu, is, o);
      id += __shfl_xor_sync(0xffffffffu, id, o);
      iq += __shfl_xor_sync(0xffffffffu, iq, o);
    }
    if (lane == 0) s_i[0][warp] = is, s_i[1][warp] = id, s_i[2][warp] = iq;
  } else {
    double ds = fs, dd = fd, dq = fq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ds += __shfl_xor_sync(0xffffffffu, ds, o);
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
      dq += __shfl_xor_sync(0xffffffffu, dq, o);
    }
    if (lane == 0) s_f[0][warp] = ds, s_f[1][warp] = dd, s_f[2][warp] = dq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t slot = ((int64_t)d * a.nblk_t + blockIdx.x) * 3;
    if constexpr (INT) {
      long long x = 0, y = 0, z = 0;
      for (int w = 0; w < kWarps; ++w) x += s_i[0][w], y += s_i[1][w], z += s_i[2][w];
      long long* o = static_cast<long long*>(a.post_part) + slot;
      o[0] = x, o[1] = y, o[2] = z;
    } else {
      double x = 0, y = 0, z = 0;
      for (int w = 0; w < kWarps; ++w) x += s_f[0][w], y += s_f[1][w], z += s_f[2][w];
      double* o = static_cast<double*>(a.post_part) + slot;
      o[0] = x, o[1] = y, o[2] = z;
    }
  }
}

template <bool INT>
cudaError_t launch_post(const DetectArgs& a, cudaStream_t s) {
  const dim3 grid((unsigned)a.nblk_t, (unsigned)a.ndm);
  switch (a.median_width) {
    case 1: post_kernel<INT, 1><<<grid, kThreads, 0, s>>>(a); break;
    case 3: post_kernel<INT, 3><<<grid, kThreads, 0, s>>>(a); break;
    case 5: post_kernel<INT, 5><<<grid, kThreads, 0, s>>>(a); break;
    case 7: post_kernel<INT, 7><<<grid, kThreads, 0, s>>>(a); break;
    case 9: post_kernel<INT, 9><<<grid, kThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Post-processed rows: sums of the post_kernel tiles (tile order, exact for
// int data), then the plain statistics or the detrending line of R11.
__device__ void row_stats_post(const DetectArgs& a, int d) {
  __shared__ double s_f[3][kThreads];
  __shared__ long long s_i[3][kThreads];
  const int64_t T = a.nout;
  double sy = 0.0, suy = 0.0, syy = 0.0;
  long long iy = 0, iuy = 0, iyy = 0;
  for (int b = threadIdx.x; b < a.nblk_t; b += kThreads) {
    // u_t = 2t - (T - 1) = 2 (t - t_c) + (2 t_c - (T - 1))
    const long long uc = 2LL * ((long long)b * kDetectT + kDetectT / 2) - (T - 1);
    const int64_t slot = ((int64_t)d * a.nblk_t + b) * 3;
    if (a.is_int) {
      const long long* o = static_cast<const long long*>(a.post_part) + slot;
      iy += o[0];
      iuy += 2 * o[1] + uc * o[0];
      iyy += o[2];
    } else {
      const double* o = static_cast<const double*>(a.post_part) + slot;
      sy += o[0];
      suy += 2.0 * o[1] + (double)uc * o[0];
      syy += o[2];
    }
  }
  s_f[0][threadIdx.x] = sy, s_f[1][threadIdx.x] = suy, s_f[2][threadIdx.x] = syy;
  s_i[0][threadIdx.x] = iy, s_i[1][threadIdx.x] = iuy, s_i[2][threadIdx.x] = iyy;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        s_f[k][threadIdx.x] += s_f[k][threadIdx.x + o];
        s_i[k][threadIdx.x] += s_i[k][threadIdx.x + o];
      }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double Sy = a.is_int ? (double)s_i[0][0] : s_f[0][0];
  const double Suy = a.is_int ? (double)s_i[1][0] : s_f[1][0];
  const double Syy = a.is_int ? (double)s_i[2][0] : s_f[2][0];
  const double Tn = (double)T;
  double m, sig, beta = 0.0;
  if (a.detrend) {
    const double Suu = (double)(((T - 1) * T * (T + 1)) / 3);
    m = __ddiv_rn(Sy, Tn);
    beta = T > 1 ? __ddiv_rn(Suy, Suu) : 0.0;
    double rss = __dsub_rn(Syy, __ddiv_rn(__dmul_rn(Sy, Sy), Tn));
    if (T > 1) rss = __dsub_rn(rss, __ddiv_rn(__dmul_rn(Suy, Suy), Suu));
    sig = __dsqrt_rn(__ddiv_rn(rss > 0.0 ? rss : 0.0, Tn));
  } else {
    m = __ddiv_rn(Sy, Tn);
    const double var = __dsub_rn(__ddiv_rn(Syy, Tn), __dmul_rn(m, m));
    sig = __dsqrt_rn(var > 0.0 ? var : 0.0);
  }
  a.row_mu[d] = m;
  a.row_sigma[d] = sig;
  a.row_beta[d] = beta;
}

__global__ void __launch_bounds__(kThreads) row_stats_kernel(DetectArgs a) {
  const int d = blockIdx.x;
  __shared__ double s_a[kThreads], s_b[kThreads];
  __shared__ long long s_ia[kThreads], s_ib[kThreads];
  if (a.median_width > 1 || a.detrend) {
    row_stats_post(a, d);
    __syncthreads();
    if (threadIdx.x != 0 || a.detrend) return;
    // plain statistics of the filtered series: the thresholds below
    const double m = a.row_mu[d], sig = a.row_sigma[d];
    const double thr = __dmul_rn(a.nsigma, sig);
    if (!(sig > 0.0)) {
      a.row_thr_f[d] = __int_as_float(0x7f800000);
      a.row_thr_i[d] = INT_MAX;
      return;
    }
    float f = (float)__dadd_rn(m, thr);
    if (passes((double)f, m, thr)) {
      for (int it = 0; it < 64; ++it) {
        const float g = nextafterf(f, -FLT_MAX);
        if (g == f || !passes((double)g, m, thr)) break;
        f = g;
      }
    } else {
      for (int it = 0; it < 64 && !passes((double)f, m, thr); ++it) f = nextafterf(f, FLT_MAX);
    }
    a.row_thr_f[d] = f;
    a.row_thr_i[d] = smallest_passing_int(m, thr);
    return;
  }
  if (a.is_int) {
    long long x = 0, y = 0;
    const longlong2* p = static_cast<const longlong2*>(a.row_part) + (int64_t)d * a.ntt;
    for (int i = threadIdx.x; i < a.ntt; i += kThreads) {
      const longlong2 v = p[i];
      x += v.x;
      y += v.y;
    }
    s_ia[threadIdx.x] = x;
    s_ib[threadIdx.x] = y;
  } else {
    double x = 0.0, y = 0.0;
    const double2* p = static_cast<const double2*>(a.row_part) + (int64_t)d * a.ntt;
    for (int i = threadIdx.x; i < a.ntt; i += kThreads) {
      const double2 v = p[i];
      x += v.x;
      y += v.y;
    }
    s_a[threadIdx.x] = x;
    s_b[threadIdx.x] = y;
  }
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      if (a.is_int) {
        s_ia[threadIdx.x] += s_ia[threadIdx.x + o];
        s_ib[threadIdx.x] += s_ib[threadIdx.x + o];
      } else {
        s_a[threadIdx.x] += s_a[threadIdx.x + o];
        s_b[threadIdx.x] += s_b[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double T = (double)a.nout;
  double m, var;
  if (a.is_int) {
    m = __ddiv_rn((double)s_ia[0], T);
    var = __dsub_rn(__ddiv_rn((double)s_ib[0], T), __dmul_rn(m, m));
  } else {
    m = __ddiv_rn(s_a[0], T);
    var = __dsub_rn(__ddiv_rn(s_b[0], T), __dmul_rn(m, m));
  }
  const double sig = __dsqrt_rn(var > 0.0 ? var : 0.0);
  a.row_mu[d] = m;
  a.row_sigma[d] = sig;
  const double thr = __dmul_rn(a.nsigma, sig);
  if (!(sig > 0.0)) {  // nothing passes
    a.row_thr_f[d] = __int_as_float(0x7f800000);  // +inf: no finite D reaches it
    a.row_thr_i[d] = INT_MAX;
    return;
  }
  // smallest float f with passes(f); the predicate is monotone in f
  float f = (float)__dadd_rn(m, thr);
  if (passes((double)f, m, thr)) {
    for (int it = 0; it < 64; ++it) {
      const float g = nextafterf(f, -FLT_MAX);
      if (g == f || !passes((double)g, m, thr)) break;
      f = g;
    }
  } else {
    for (int it = 0; it < 64 && !passes((double)f, m, thr); ++it) f = nextafterf(f, FLT_MAX);
  }
  a.row_thr_f[d] = f;
  a.row_thr_i[d] = smallest_passing_int(m, thr);
}

// the series the detection reads: the median-filtered one, else D
__device__ __forceinline__ const void* det_series(const DetectArgs& a) { return a.median_width > 1 ? a.M : a.D; }

// Detrended test of one sample in FP32: 1 = pass, 0 = fail, 2 = undecided.
// The FP32 residual y - (mean + beta u) is within a few units in 2^-24 of
// |y| + |mean| + |beta u| + thr of the exact one; the margin below is far
// wider, so only samples inside it are undecided and take the binary64 test
// (in the oracle's operation order).  u is exact in FP32 (|u| < 2^24).
__device__ __forceinline__ int detrend_hit32(float y, float u, float m32, float b32, float thr32) {
  const float bu = b32 * u;
  const float r32 = y - (m32 + bu);
  const float guard = 1e-5f * (fabsf(y) + fabsf(m32) + fabsf(bu) + thr32);
  if (r32 > thr32 + guard) return 1;
  if (r32 < thr32 - guard) return 0;
  return 2;
}

__global__ void __launch_bounds__(kThreads) detect_count(DetectArgs a) {
  const int d = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * kDetectT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the CTA reads row d of the series in [0, nout) and writes its words of
  // row d of the hit bitmap
  if (!in_bounds(0, a.nout, a.dpitch, a.status) || !in_bounds((int64_t)d * a.dpitch, a.nout, a.d_elems, a.status) ||
      !in_bounds((int64_t)d * a.hit_pitch, a.hit_pitch, a.hit_elems, a.status))
    return;
  const float tf = a.row_thr_f[d];
  const int ti = a.row_thr_i[d];
  const void* S = det_series(a);
  // detrended rows: line and threshold (sigma = 0: nothing passes)
  double mean = 0.0, beta = 0.0, thr = 0.0;
  float m32 = 0.f, b32 = 0.f, thr32 = 0.f;
  bool live = true;
  if (a.detrend) {
    mean = a.row_mu[d];
    beta = a.row_beta[d];
    const double sig = a.row_sigma[d];
    live = sig > 0.0;
    thr = __dmul_rn(a.nsigma, sig);
    m32 = (float)mean, b32 = (float)beta, thr32 = (float)thr;
  }
  int cnt = 0;
  // thread handles 4 runs of 4 consecutive samples: t = t0 + 1024 r + 4 tid + e
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t tb = t0 + 1024 * r + 4 * threadIdx.x;
    bool hit[4] = {false, false, false, false};
    if (a.detrend) {
      if (live && tb < a.nout) {
        float y[4];
        const int64_t base = (int64_t)d * a.dpitch + tb;
        if (tb + 3 < a.nout) {
          if (a.is_int) {
            const int4 v = *reinterpret_cast<const int4*>(static_cast<const int*>(S) + base);
            y[0] = (float)v.x, y[1] = (float)v.y, y[2] = (float)v.z, y[3] = (float)v.w;
          } else {
            const float4 v = *reinterpret_cast<const float4*>(static_cast<const float*>(S) + base);
            y[0] = v.x, y[1] = v.y, y[2] = v.z, y[3] = v.w;
          }
        } else {
          for (int e = 0; e < 4; ++e)
            y[e] = tb + e < a.nout ? (a.is_int ? (float)static_cast<const int*>(S)[base + e]
                                               : static_cast<const float*>(S)[base + e])
                                   : 0.f;
        }
        const float u0 = (float)(2 * tb - (a.nout - 1));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (tb + e >= a.nout) break;
          const int h = detrend_hit32(y[e], u0 + 2.f * e, m32, b32, thr32);
          if (h == 2) {
            const double v = a.is_int ? (double)static_cast<const int*>(S)[base + e]
                                      : (double)static_cast<const float*>(S)[base + e];
            hit[e] = residual(v, mean, beta, (double)(2 * (tb + e) - (a.nout - 1))) >= thr;
          } else {
            hit[e] = h == 1;
          }
        }
      }
    } else if (a.is_int) {
      const int* row = static_cast<const int*>(S) + (int64_t)d * a.dpitch;
      if (tb + 3 < a.nout) {
        const int4 v = *reinterpret_cast<const int4*>(row + tb);
        hit[0] = v.x >= ti, hit[1] = v.y >= ti, hit[2] = v.z >= ti, hit[3] = v.w >= ti;
      } else {
        for (int e = 0; e < 4; ++e) hit[e] = tb + e < a.nout && row[tb + e] >= ti;
      }
    } else {
      const float* row = static_cast<const float*>(S) + (int64_t)d * a.dpitch;
      if (tb + 3 < a.nout) {
        const float4 v = *reinterpret_cast<const float4*>(row + tb);
        hit[0] = v.x >= tf, hit[1] = v.y >= tf, hit[2] = v.z >= tf, hit[3] = v.w >= tf;
      } else {
        for (int e = 0; e < 4; ++e) hit[e] = tb + e < a.nout && row[tb + e] >= tf;
      }
    }
    // bit (t - t0) of the CTA's 128 words; 4 consecutive samples per lane
    const unsigned nib = (unsigned)hit[0] | ((unsigned)hit[1] << 1) | ((unsigned)hit[2] << 2) |
                         ((unsigned)hit[3] << 3);
    // lanes 8k..8k+7 fill one 32-bit word
    unsigned wv = nib << (4 * (lane & 7));
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) wv |= __shfl_xor_sync(0xffffffffu, wv, o);
    const int64_t word = (t0 + 1024 * r + 4 * (threadIdx.x & ~7)) >> 5;
    if ((lane & 7) == 0 && word < a.hit_pitch) a.hit_bits[(int64_t)d * a.hit_pitch + word] = wv;
    cnt += __popc(nib);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __shared__ int s_cnt[kWarps];
  if (lane == 0) s_cnt[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < kWarps; ++w) tot += s_cnt[w];
    a.blk_count[(int64_t)d * a.nblk_t + blockIdx.x] = (uint32_t)tot;
  }
}

__global__ void __launch_bounds__(1024) detect_scan(DetectArgs a, int nblk) {
  __shared__ unsigned long long s[1024];
  const int per = (nblk + 1023) / 1024;
  const int lo = threadIdx.x * per;
  const int hi = lo + per < nblk ? lo + per : nblk;
  // the thread's counts eight at a time, their loads issued together
  unsigned long long sum = 0;
  for (int i0 = lo; i0 < hi; i0 += 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = i0 + u < hi ? a.blk_count[i0 + u] : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += v[u];
  }
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned long long v = threadIdx.x >= o ? s[threadIdx.x - o] : 0ull;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = s[threadIdx.x] - sum;  // exclusive prefix
  for (int i0 = lo; i0 < hi; i0 += 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = i0 + u < hi ? a.blk_count[i0 + u] : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (i0 + u < hi) a.blk_off[i0 + u] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
      run += v[u];
    }
  }
  if (threadIdx.x == 1023) *a.n_total = s[1023];
}

// Thread (warp w, lane l) owns hit word j*8 + w of the CTA (words in t order).
__global__ void __launch_bounds__(kThreads) detect_write(DetectArgs a) {
  const int d = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * kDetectT;
  const uint32_t cnt = a.blk_count[(int64_t)d * a.nblk_t + blockIdx.x];
  if (cnt == 0) return;
  const uint64_t base = a.blk_off[(int64_t)d * a.nblk_t + blockIdx.x];
  if (base >= (uint64_t)a.cap) return;
  if (!in_bounds((int64_t)d * a.dpitch, a.nout, a.d_elems, a.status) ||
      !in_bounds((int64_t)d * a.hit_pitch, a.hit_pitch, a.hit_elems, a.status))
    return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ uint32_t s_pre[kPer * kWarps];
  uint32_t words[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int64_t word = (t0 >> 5) + j * kWarps + warp;
    words[j] = word < a.hit_pitch ? a.hit_bits[(int64_t)d * a.hit_pitch + word] : 0u;
    if (lane == 0) s_pre[j * kWarps + warp] = __popc(words[j]);
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan over the 128 word counts, in t order
    uint32_t v[4], tot = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = s_pre[lane * 4 + q], tot += v[q];
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += n;
    }
    uint32_t run = inc - tot;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t c = v[q];
      s_pre[lane * 4 + q] = run;
      run += c;
    }
  }
  __syncthreads();
  const double mu = a.row_mu[d], sigma = a.row_sigma[d];
  const double beta = a.detrend ? a.row_beta[d] : 0.0;
  const void* S = det_series(a);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t w = words[j];
    if ((w >> lane) & 1u) {
      const uint32_t rank = s_pre[j * kWarps + warp] + __popc(w & ((1u << lane) - 1u));
      const uint64_t pos = base + rank;
      const int64_t t = t0 + 32 * ((int64_t)j * kWarps + warp) + lane;
      if (pos < (uint64_t)a.cap && in_bounds(t, 1, a.nout, a.status)) {
        const double v = a.is_int ? (double)static_cast<const int*>(S)[(int64_t)d * a.dpitch + t]
                                  : (double)static_cast<const float*>(S)[(int64_t)d * a.dpitch + t];
        tp_candidate r;
        r.beam = a.beam;
        r.dm_idx = d;
        r.t_abs = *a.t0_abs + t;
        const double res = a.detrend ? residual(v, mu, beta, (double)(2 * t - (a.nout - 1))) : __dsub_rn(v, mu);
        r.snr = (float)__ddiv_rn(res, sigma);
        r.value = (float)v;
        a.cand[pos] = r;
      }
    }
  }
}

// Stream-ordered export of a beam's candidate list: the count found and the
// first min(found, beam capacity, cap) records, copied as 8-byte words by a
// grid-stride loop into memory the device can write (page-locked host memory
// or device memory); the beam's status word goes along with them and is
// cleared for the next block.
__global__ void __launch_bounds__(kThreads) export_candidates_kernel(const tp_candidate* __restrict__ cand,
                                                                    const unsigned long long* n_total, int beam_cap,
                                                                    int* status, tp_candidate* out, int cap,
                                                                    unsigned long long* out_count, int* out_status) {
  static_assert(sizeof(tp_candidate) == 24, "three 8-byte words per record");
  const unsigned long long tot = *n_total;
  const unsigned long long kept = tot < (unsigned long long)beam_cap ? tot : (unsigned long long)beam_cap;
  const int64_t n = (int64_t)(kept < (unsigned long long)cap ? kept : (unsigned long long)cap);
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(cand);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(out);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *out_count = tot;
    const int st = atomicExch(status, 0);
    if (out_status) *out_status = st;
  }
}

}  // namespace

cudaError_t launch_detect(const DetectArgs& a, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (a.median_width > 1 || a.detrend) {
    e = a.is_int ? launch_post<true>(a, s) : launch_post<false>(a, s);
    if (e != cudaSuccess) return e;
  }
  row_stats_kernel<<<a.ndm, kThreads, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)a.nblk_t, (unsigned)a.ndm);
  detect_count<<<grid, kThreads, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  detect_scan<<<1, 1024, 0, s>>>(a, a.nblk_t * a.ndm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  detect_write<<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_export_candidates(const tp_candidate* cand, const unsigned long long* n_total, int beam_cap,
                                     int* status, tp_candidate* out, int cap, unsigned long long* out_count,
                                     int* out_status, int grid, cudaStream_t s) {
  export_candidates_kernel<<<(unsigned)(grid > 0 ? grid : 1), kThreads, 0, s>>>(cand, n_total, beam_cap, status, out,
                                                                               cap, out_count, out_status);
  return cudaGetLastError();
}

}  // namespace tp
