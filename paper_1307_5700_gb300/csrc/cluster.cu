// Clustering and classification of a block's detections (Sec. 2.3, after the
// n-sigma threshold): DBSCAN with a per-dimension box neighbourhood, then the
// DM-SNR classification against Eq. 3-4 for every cluster.
//
// Input: the beam's candidate records in (d, t) order (the first
// min(n_total, capacity) of them).  Neighbourhood of p: the records q with
// |d_q - d_p| <= dm_eps, |t_q - t_p| <= t_eps, |snr_q - snr_p| <= snr_eps
// (p included); core points have >= min_pts neighbours.  Clusters are the
// connected groups of core points, found with a lock-free union-find that
// always links the higher root under the lower, so every group's root is its
// lowest-index core point; a border point (not core, with a core neighbour)
// joins the cluster of its lowest-index core neighbour; clusters are
// numbered in the order of their roots.  The result is unique, so the oracle
// reproduces it exactly.  (The paper runs FDBSCAN, an approximation that
// saves region queries on a CPU; on the sorted records a region query is two
// binary searches per DM trial, so the exact clustering is kept.)
//
// Classification, one CTA per cluster at a time: the largest SNR per DM trial (the
// DM-SNR signature), its centred k-trial moving average, the trial d* with
// the most detections (below dm_min: broadband RFI), the width there, the
// signature normalised by its maximum, Eq. 3-4 for the DM errors to d*, and
// the RMSE of the two; a candidate when not broadband RFI and the RMSE is at
// most rmse_max.
#include <climits>
#include <cstdint>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int cand_count(const ClusterArgs& a) {
  const unsigned long long n = *a.n_total;
  return n < (unsigned long long)a.cap ? (int)n : a.cap;
}

// first index in [lo, hi) whose t_abs is >= t (records of one DM row)
__device__ __forceinline__ int lower_t(const tp_candidate* c, int lo, int hi, int64_t t) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (c[mid].t_abs < t) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Calls f(q) for every neighbour q of p (p included), in index order.
template <typename F>
__device__ __forceinline__ void for_neighbours(const ClusterArgs& a, int p, F f) {
  const tp_candidate cp = a.cand[p];
  const int d0 = cp.dm_idx - a.dm_eps < 0 ? 0 : cp.dm_idx - a.dm_eps;
  const int d1 = cp.dm_idx + a.dm_eps > a.ndm - 1 ? a.ndm - 1 : cp.dm_idx + a.dm_eps;
  for (int d = d0; d <= d1; ++d) {
    const int hi = a.row_start[d + 1];
    for (int q = lower_t(a.cand, a.row_start[d], hi, cp.t_abs - a.t_eps); q < hi; ++q) {
      const tp_candidate cq = a.cand[q];
      if (cq.t_abs > cp.t_abs + a.t_eps) break;
      if (fabsf(cq.snr - cp.snr) <= a.snr_eps) f(q);
    }
  }
}

__global__ void cl_rows(ClusterArgs a) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d > a.ndm) return;
  const int n = cand_count(a);
  int lo = 0, hi = n;  // first record with dm_idx >= d
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a.cand[mid].dm_idx < d) lo = mid + 1;
    else hi = mid;
  }
  a.row_start[d] = lo;
  if (d == 0) *a.n_clusters = 0;
}

__global__ void cl_core(ClusterArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cand_count(a)) return;
  int cnt = 0;
  for_neighbours(a, p, [&](int) { ++cnt; });
  a.core[p] = cnt >= a.min_pts ? 1 : 0;
  a.parent[p] = p;
}

// Root of p's group, halving the path on the way (a non-root's parent is
// set to its grandparent: an ancestor, so concurrent finds and the roots'
// compare-and-swap links stay valid).
__device__ __forceinline__ int find_root(int* parent, int p) {
  int r = p;
  for (int it = 0; it < (1 << 24); ++it) {  // bounded: a root is reached in fewer steps than points
    const int q = parent[r];
    if (q == r) return r;
    const int g = parent[q];
    if (g != q) parent[r] = g;
    r = g;
  }
  return r;
}

// union of the groups of u and v: the higher root is linked under the lower
__device__ void unite(int* parent, int u, int v) {
  for (int it = 0; it < (1 << 24); ++it) {
    const int ru = find_root(parent, u), rv = find_root(parent, v);
    if (ru == rv) return;
    const int hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
    if (atomicCAS(&parent[hi], hi, lo) == hi) return;
  }
}

// One warp per core point p (a fixed grid strides over the points), its
// lanes splitting p's neighbours q < p: those lie in the trials up to p's
// own (records are in (d, t) order), the links to higher neighbours are
// made by those neighbours' warps.
__global__ void __launch_bounds__(kThreads) cl_union(ClusterArgs a) {
  const int n = cand_count(a);
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (kThreads / 32);
  for (int p = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); p < n; p += warps) {
    if (!a.core[p]) continue;
    const tp_candidate cp = a.cand[p];
    const int d0 = cp.dm_idx - a.dm_eps < 0 ? 0 : cp.dm_idx - a.dm_eps;
    int rp = find_root(a.parent, p);  // may go stale; unite() re-checks
    for (int d = d0; d <= cp.dm_idx; ++d) {
      const int hi = d == cp.dm_idx ? p : a.row_start[d + 1];
      for (int q = lower_t(a.cand, a.row_start[d], hi, cp.t_abs - a.t_eps) + lane; q < hi; q += 32) {
        const tp_candidate cq = a.cand[q];
        if (cq.t_abs > cp.t_abs + a.t_eps) break;
        if (fabsf(cq.snr - cp.snr) <= a.snr_eps && a.core[q] && find_root(a.parent, q) != rp) {
          unite(a.parent, p, q);
          rp = find_root(a.parent, p);
        }
      }
    }
  }
}

// root of every point's cluster (-1: noise)
__global__ void cl_assign(ClusterArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cand_count(a)) return;
  int r = -1;
  if (a.core[p]) {
    r = find_root(a.parent, p);
  } else {
    int best = -1;
    for_neighbours(a, p, [&](int q) {
      if (best < 0 && a.core[q]) best = q;  // neighbours arrive in index order
    });
    if (best >= 0) r = find_root(a.parent, best);
  }
  a.root[p] = r;
}

// cluster numbers: rank of every root among the roots (one CTA)
__global__ void __launch_bounds__(1024) cl_number(ClusterArgs a) {
  const int n = cand_count(a);
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
  int cnt = 0;
  for (int p = lo; p < hi; ++p) cnt += (a.core[p] && a.parent[p] == p) ? 1 : 0;
  __shared__ int s[1024];
  s[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s[threadIdx.x] - cnt;
  for (int p = lo; p < hi; ++p)
    if (a.core[p] && a.parent[p] == p) a.rank[p] = run++;
  if (threadIdx.x == 1023) *a.n_clusters = s[1023] < a.max_clusters ? s[1023] : a.max_clusters;
  if (threadIdx.x == 1023) *a.truncated = s[1023] > a.max_clusters ? 1 : 0;
}

__global__ void cl_label(ClusterArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cand_count(a)) return;
  int l = -1;
  if (a.root[p] >= 0) {
    const int k = a.rank[a.root[p]];
    if (k < a.max_clusters) {
      l = k;
      atomicAdd(&a.cl_count[k], 1);
    }
  }
  a.label[p] = l;
}

__global__ void __launch_bounds__(1024) cl_offsets(ClusterArgs a) {
  const int n = *a.n_clusters;
  const int per = (n + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
  int cnt = 0;
  for (int k = lo; k < hi; ++k) cnt += a.cl_count[k];
  __shared__ int s[1024];
  s[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s[threadIdx.x] - cnt;
  for (int k = lo; k < hi; ++k) {
    a.cl_offset[k] = run;
    a.cl_cursor[k] = 0;
    run += a.cl_count[k];
  }
  if (threadIdx.x == 1023) a.cl_offset[n] = s[1023];
}

__global__ void cl_scatter(ClusterArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cand_count(a)) return;
  const int l = a.label[p];
  if (l >= 0) a.order[a.cl_offset[l] + atomicAdd(&a.cl_cursor[l], 1)] = p;
}

// order-preserving integer key of a float (for atomicMax)
__device__ __forceinline__ int fkey(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float fval(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__device__ double eq3(double ddm, double width_ms, double bw_mhz, double f_ghz) {
  const double z = 6.91e-3 * fabs(ddm) * bw_mhz / (width_ms * (f_ghz * f_ghz * f_ghz));
  if (z == 0.0) return 1.0;
  return sqrt(3.141592653589793) / 2.0 * erf(z) / z;
}

// sum or maximum over the CTA (every thread gets the result)
template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double* s_red) {
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? (w > v ? w : v) : v + w;
  }
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = s_red[0];
  for (int i = 1; i < kThreads / 32; ++i) v = MAX ? (s_red[i] > v ? s_red[i] : v) : v + s_red[i];
  __syncthreads();
  return v;
}

// One cluster: dynamic shared memory holds [ndm] doubles (the smoothed
// signature), then [ndm] max-SNR keys and [ndm] detection counts.
__device__ void classify_one(const ClusterArgs& a, int k, double* s_v, int* s_sig, int* s_cnt) {
  const int b0 = a.cl_offset[k], b1 = a.cl_offset[k + 1];
  __shared__ int s_dlo, s_dhi, s_smax;
  __shared__ long long s_t0, s_t1, s_w0, s_w1;
  __shared__ unsigned long long s_best;
  __shared__ double s_red[kThreads / 32];
  if (threadIdx.x == 0) {
    s_dlo = INT_MAX, s_dhi = -1, s_smax = fkey(-INFINITY);
    s_t0 = LLONG_MAX, s_t1 = LLONG_MIN, s_w0 = LLONG_MAX, s_w1 = LLONG_MIN;
    s_best = 0;
  }
  __syncthreads();
  for (int i = b0 + threadIdx.x; i < b1; i += kThreads) {
    const tp_candidate c = a.cand[a.order[i]];
    atomicMin(&s_dlo, c.dm_idx);
    atomicMax(&s_dhi, c.dm_idx);
    atomicMax(&s_smax, fkey(c.snr));
    atomicMin(&s_t0, (long long)c.t_abs);
    atomicMax(&s_t1, (long long)c.t_abs);
  }
  __syncthreads();
  const int lo = s_dlo, span = s_dhi - s_dlo + 1;
  for (int i = threadIdx.x; i < span; i += kThreads) s_sig[i] = fkey(0.f), s_cnt[i] = 0;
  __syncthreads();
  for (int i = b0 + threadIdx.x; i < b1; i += kThreads) {
    const tp_candidate c = a.cand[a.order[i]];
    atomicMax(&s_sig[c.dm_idx - lo], fkey(c.snr));
    atomicAdd(&s_cnt[c.dm_idx - lo], 1);
  }
  __syncthreads();
  // d*: the most detections, ties to the lowest trial
  for (int i = threadIdx.x; i < span; i += kThreads)
    if (s_cnt[i] > 0)
      atomicMax(&s_best, ((unsigned long long)s_cnt[i] << 32) | (unsigned)(INT_MAX - i));
  __syncthreads();
  const int ds = lo + (INT_MAX - (int)(unsigned)(s_best & 0xffffffffu));
  for (int i = b0 + threadIdx.x; i < b1; i += kThreads) {
    const tp_candidate c = a.cand[a.order[i]];
    if (c.dm_idx == ds) {
      atomicMin(&s_w0, (long long)c.t_abs);
      atomicMax(&s_w1, (long long)c.t_abs);
    }
  }
  __syncthreads();
  const double width_ms = (double)(s_w1 - s_w0 + 1) * a.t_samp * 1e3;
  // centred moving average of the signature (each trial's window summed in
  // DM order), its maximum, and the RMSE against Eq. 3
  const int h = a.smooth / 2;
  double vmax = 0.0;
  for (int i = threadIdx.x; i < span; i += kThreads) {
    const int p0 = i - h < 0 ? 0 : i - h, p1 = i + h + 1 > span ? span : i + h + 1;
    double v = 0.0;
    for (int j = p0; j < p1; ++j) v += (double)fval(s_sig[j]);
    v /= (double)(p1 - p0);
    s_v[i] = v;
    vmax = v > vmax ? v : vmax;
  }
  const double smax = block_reduce<true>(vmax, s_red);
  const double dm_star = a.dm[ds];
  double ss = 0.0;
  for (int i = threadIdx.x; i < span; i += kThreads) {
    const double r = s_v[i] / smax - eq3(a.dm[lo + i] - dm_star, width_ms, a.bw_mhz, a.f_ghz);
    ss += r * r;
  }
  ss = block_reduce<false>(ss, s_red);
  if (threadIdx.x == 0) {
    const double rmse = sqrt(ss / (double)span);
    const bool broadband = dm_star < a.dm_min;
    tp_cluster r;
    r.label = k;
    r.n = b1 - b0;
    r.d_lo = lo;
    r.d_hi = s_dhi;
    r.d_star = ds;
    r.flags = (broadband ? 2 : 0) | ((!broadband && rmse <= a.rmse_max) ? 1 : 0);
    r.t_first = s_t0;
    r.t_last = s_t1;
    r.snr_max = fval(s_smax);
    r.width_ms = (float)width_ms;
    r.rmse = (float)rmse;
    r.reserved = 0.f;
    a.clusters[k] = r;
  }
  __syncthreads();
}

// A fixed grid strides over the clusters, one cluster per CTA at a time.
__global__ void __launch_bounds__(kThreads) cl_classify(ClusterArgs a) {
  extern __shared__ double s_dyn[];
  double* s_v = s_dyn;
  int* s_sig = reinterpret_cast<int*>(s_dyn + a.ndm);
  int* s_cnt = s_sig + a.ndm;
  const int n = *a.n_clusters;
  for (int k = blockIdx.x; k < n; k += gridDim.x) classify_one(a, k, s_v, s_sig, s_cnt);
}

}  // namespace

cudaError_t launch_cluster(const ClusterArgs& a, cudaStream_t s) {
  const unsigned gp = (unsigned)((a.cap + kThreads - 1) / kThreads);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.cl_count, 0, sizeof(int) * (size_t)a.max_clusters, s);
  if (e != cudaSuccess) return e;
  cl_rows<<<(a.ndm + 1 + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
  cl_core<<<gp, kThreads, 0, s>>>(a);
  cl_union<<<8 * sms, kThreads, 0, s>>>(a);
  cl_assign<<<gp, kThreads, 0, s>>>(a);
  cl_number<<<1, 1024, 0, s>>>(a);
  cl_label<<<gp, kThreads, 0, s>>>(a);
  cl_offsets<<<1, 1024, 0, s>>>(a);
  cl_scatter<<<gp, kThreads, 0, s>>>(a);
  const size_t sm = (sizeof(double) + 2 * sizeof(int)) * (size_t)a.ndm;
  e = cudaFuncSetAttribute(cl_classify, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = a.max_clusters < 4 * sms ? a.max_clusters : 4 * sms;
  cl_classify<<<(unsigned)grid, kThreads, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tp
