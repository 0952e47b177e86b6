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
#include <cfloat>
#include <climits>
#include <cstdint>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPer = kDetectT / kThreads;  // 16 samples per thread

__device__ __forceinline__ bool passes(double v, double mu, double thr) { return __dsub_rn(v, mu) >= thr; }

__global__ void __launch_bounds__(kThreads) row_stats_kernel(DetectArgs a) {
  const int d = blockIdx.x;
  __shared__ double s_a[kThreads], s_b[kThreads];
  __shared__ long long s_ia[kThreads], s_ib[kThreads];
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
  // smallest int i with passes(i)
  const double c = ceil(__dadd_rn(m, thr));
  long long i = c > 2147483647.0 ? 2147483647LL : (c < -2147483648.0 ? -2147483648LL : (long long)c);
  while (i > INT_MIN && passes((double)(i - 1), m, thr)) --i;
  while (i < INT_MAX && !passes((double)i, m, thr)) ++i;
  a.row_thr_i[d] = (int)i;
}

__global__ void __launch_bounds__(kThreads) detect_count(DetectArgs a) {
  const int d = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * kDetectT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float tf = a.row_thr_f[d];
  const int ti = a.row_thr_i[d];
  int cnt = 0;
  // thread handles 4 runs of 4 consecutive samples: t = t0 + 1024 r + 4 tid + e
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t tb = t0 + 1024 * r + 4 * threadIdx.x;
    bool hit[4] = {false, false, false, false};
    if (a.is_int) {
      const int* row = static_cast<const int*>(a.D) + (int64_t)d * a.dpitch;
      if (tb + 3 < a.nout) {
        const int4 v = *reinterpret_cast<const int4*>(row + tb);
        hit[0] = v.x >= ti, hit[1] = v.y >= ti, hit[2] = v.z >= ti, hit[3] = v.w >= ti;
      } else {
        for (int e = 0; e < 4; ++e) hit[e] = tb + e < a.nout && row[tb + e] >= ti;
      }
    } else {
      const float* row = static_cast<const float*>(a.D) + (int64_t)d * a.dpitch;
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
  unsigned long long sum = 0;
  for (int i = lo; i < hi; ++i) sum += a.blk_count[i];
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    unsigned long long v = threadIdx.x >= o ? s[threadIdx.x - o] : 0ull;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = s[threadIdx.x] - sum;  // exclusive prefix
  for (int i = lo; i < hi; ++i) {
    const uint32_t c = a.blk_count[i];
    a.blk_off[i] = (uint32_t)(run < 0xffffffffull ? run : 0xffffffffull);
    run += c;
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
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const uint32_t w = words[j];
    if ((w >> lane) & 1u) {
      const uint32_t rank = s_pre[j * kWarps + warp] + __popc(w & ((1u << lane) - 1u));
      const uint64_t pos = base + rank;
      if (pos < (uint64_t)a.cap) {
        const int64_t t = t0 + 32 * ((int64_t)j * kWarps + warp) + lane;
        const double v = a.is_int ? (double)static_cast<const int*>(a.D)[(int64_t)d * a.dpitch + t]
                                  : (double)static_cast<const float*>(a.D)[(int64_t)d * a.dpitch + t];
        tp_candidate r;
        r.beam = a.beam;
        r.dm_idx = d;
        r.t_abs = *a.t0_abs + t;
        r.snr = (float)__ddiv_rn(__dsub_rn(v, mu), sigma);
        r.value = (float)v;
        a.cand[pos] = r;
      }
    }
  }
}

}  // namespace

cudaError_t launch_detect(const DetectArgs& a, cudaStream_t s) {
  row_stats_kernel<<<a.ndm, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
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

}  // namespace tp
