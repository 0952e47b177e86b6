// A6-A7: per-DM series statistics (normalisation of Sec. 2.2.3) and the
// n-sigma detection of Sec. 2.3, compacted on the device.
//
//   mu_d = sum_t D / T,  sigma_d^2 = sum_t D^2 / T - mu_d^2   (population)
//   candidate (d, t)  <=>  sigma_d > 0  and  D[d][t] - mu_d >= nsigma * sigma_d
//
// The sums come from the per-(DM, time-tile) partials written by the
// dedispersion epilogue (exact int64 for 8-bit data).  Compaction is
// deterministic and ordered by (d, t) without a sort:
//   count : one CTA per (d, 4096 samples) evaluates the predicate, writes one
//           hit bit per sample and the CTA's hit count;
//   scan  : one CTA turns the counts into offsets (row-major in (d, t-block));
//   write : each CTA ranks its hits in t order (ballots + a 128-entry scan) and
//           writes records at offset + rank, keeping those below the capacity.
#include <cstdint>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPer = kDetectT / kThreads;  // 16 samples per thread

// Row statistics from the partials; every CTA of the row computes the same
// values in the same order.
__device__ void row_stats(const DetectArgs& a, int d, double* mu, double* sigma) {
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
  const double T = (double)a.nout;
  double m, var;
  if (a.is_int) {
    m = __ddiv_rn((double)s_ia[0], T);
    var = __dsub_rn(__ddiv_rn((double)s_ib[0], T), __dmul_rn(m, m));
  } else {
    m = __ddiv_rn(s_a[0], T);
    var = __dsub_rn(__ddiv_rn(s_b[0], T), __dmul_rn(m, m));
  }
  *mu = m;
  *sigma = __dsqrt_rn(var > 0.0 ? var : 0.0);
  __syncthreads();
}

__device__ __forceinline__ double value_at(const DetectArgs& a, int d, int64_t t) {
  if (a.is_int) return (double)static_cast<const int*>(a.D)[(int64_t)d * a.dpitch + t];
  return (double)static_cast<const float*>(a.D)[(int64_t)d * a.dpitch + t];
}

__global__ void __launch_bounds__(kThreads) detect_count(DetectArgs a) {
  const int d = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * kDetectT;
  double mu, sigma;
  row_stats(a, d, &mu, &sigma);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.row_mu[d] = mu;
    a.row_sigma[d] = sigma;
  }
  const double thr = __dmul_rn(a.nsigma, sigma);
  const bool live = sigma > 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cnt = 0;
#pragma unroll 4
  for (int j = 0; j < kPer; ++j) {
    const int64_t t = t0 + (int64_t)j * kThreads + threadIdx.x;
    bool hit = false;
    if (live && t < a.nout) hit = __dsub_rn(value_at(a, d, t), mu) >= thr;
    const unsigned bits = __ballot_sync(0xffffffffu, hit);
    const int64_t word = (t0 >> 5) + j * kWarps + warp;
    if (lane == 0 && word < a.hit_pitch) a.hit_bits[(int64_t)d * a.hit_pitch + word] = bits;
    cnt += __popc(bits);
  }
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
        const int64_t t = t0 + (int64_t)j * kThreads + threadIdx.x;
        const double v = value_at(a, d, t);
        tp_candidate r;
        r.beam = a.beam;
        r.dm_idx = d;
        r.t_abs = a.t0_abs + t;
        r.snr = (float)__ddiv_rn(__dsub_rn(v, mu), sigma);
        r.value = (float)v;
        a.cand[pos] = r;
      }
    }
  }
}

}  // namespace

cudaError_t launch_detect(const DetectArgs& a, cudaStream_t s) {
  dim3 grid((unsigned)a.nblk_t, (unsigned)a.ndm);
  detect_count<<<grid, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  detect_scan<<<1, 1024, 0, s>>>(a, a.nblk_t * a.ndm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  detect_write<<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tp
