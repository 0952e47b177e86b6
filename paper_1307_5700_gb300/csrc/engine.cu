// C ABI: engine, plans, beams and the per-block pipeline (see tp_dedisp.h).
//
// Host-side runtime: device memory is allocated once per plan / beam and kept
// resident (the overlap window, statistics, masks, series and candidate
// buffers of every beam), admission is by device-memory footprint, and every
// step of a block is issued asynchronously on the beam's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tp_common.cuh"

namespace tp {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

const char* last_error_cstr() { return g_last_error.c_str(); }

int cuda_error(cudaError_t err, const char* what) {
  return set_error(TP_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(err), cudaGetErrorName(err));
}

size_t dtype_size(int dtype) {
  switch (dtype) {
    case TP_U8: return 1;
    case TP_F16:
    case TP_BF16: return 2;
    case TP_F32:
    case TP_C16: return 4;
    default: return 0;
  }
}

// bytes per sample of the staged series y (A4 output) in the format of kernel
// shape format `fmt`: FP32 y (FP32 data, or 16-bit float data staged as
// x~ - b in FP32), the stored samples x~ in their own 16-bit format, or 8-bit
// samples widened to 16-bit integers
int staged_bytes_fmt(int fmt) { return fmt == 4 ? 4 : 2; }

// the kernel-shape staging formats (KernelShape::FMT) a dtype can use: its
// own, and FP32 staging for 16-bit float data
int staged_format(int dtype) { return dtype == TP_F32 || dtype == TP_C16 ? 4 : (dtype == TP_U8 ? 3 : 2); }
bool format_ok(int dtype, int fmt) {
  return fmt == staged_format(dtype) || (fmt == 4 && (dtype == TP_F16 || dtype == TP_BF16));
}

// bytes per sample the staged series buffer is allocated with (room for
// every format the dtype can use)
int staged_bytes_alloc(int dtype) { return dtype == TP_U8 ? 2 : 4; }

// Nearest value of a 16-bit storage format (ties to even), from the format's
// definition; the same rule the statistics kernel applies on the device.
static double round_to_format(double v, int sig, int emin, double maxv) {
  if (v == 0.0 || !std::isfinite(v)) return v;
  const double a = std::fabs(v);
  int e;
  std::frexp(a, &e);
  int qexp = e - sig;
  if (qexp < emin - sig + 1) qexp = emin - sig + 1;
  const double q = std::ldexp(1.0, qexp);
  double r = std::nearbyint(a / q) * q;
  if (r > maxv) r = INFINITY;
  return std::copysign(r, v);
}

// Bit pattern of a value already representable in the 16-bit format.
unsigned short storage_bits_host(int dtype, double mu) {
  if (dtype == TP_BF16) {
    const float f = (float)round_to_format(mu, 8, -126, 3.3895313892515355e38);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (unsigned short)(u >> 16);
  }
  const double r = round_to_format(mu, 11, -14, 65504.0);
  const unsigned short sign = std::signbit(r) ? 0x8000 : 0;
  const double a = std::fabs(r);
  if (a == 0.0) return sign;
  if (std::isinf(a)) return sign | 0x7c00;
  int e;
  std::frexp(a, &e);                       // a = m 2^e, m in [1/2, 1)
  if (e - 1 >= -14)                        // normal: a = (1 + f) 2^(e - 1)
    return sign | (unsigned short)((e - 1 + 15) << 10) |
           (unsigned short)(std::ldexp(a, 11 - e) - 1024.0);
  return sign | (unsigned short)std::ldexp(a, 24);  // subnormal: a = m 2^-24
}

}  // namespace tp

using namespace tp;

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr size_t kBatchBytes = 512 * 1024;  // batch arguments of up to ~2000 beams
constexpr size_t kMaxBatchGroups = 64;        // kernel-shape groups (launches) of one batch

enum BeamState { kEmpty = 0, kReady = 1, kDedispersed = 2, kDetected = 3 };

struct Beam {
  tp_engine* e = nullptr;
  const tp_plan* plan = nullptr;
  int id = -1;
  int B = 0;         // block length
  int cap = 0;       // candidate capacity
  int64_t pitch = 0; // window row pitch (elements)
  int nchunk_max = 0;
  int ntt_max = 0;
  int nblk_max = 0;
  int64_t hit_pitch = 0;
  int64_t dpitch = 0;
  cudaStream_t stream = nullptr;
  bool own_event = false;
  cudaEvent_t ev_detect = nullptr;  // the beam's last detection finished
  cudaEvent_t ev_pushed = nullptr;  // the beam's last push finished (its own stream)
  // prefetch of the next block (tp_prefetch_block): host -> device copy of its
  // new samples into the window the block after the current one will use, on
  // a copy stream of the beam's own
  cudaStream_t pf_stream = nullptr;
  cudaEvent_t ev_win_free = nullptr;  // the last push copied its overlap tail out of the other window
  cudaEvent_t ev_pf = nullptr;        // the pending prefetch's copy finished
  bool pf_pending = false;
  int pf_nsamp = 0;
  // device buffers
  void* win[2] = {nullptr, nullptr};
  void* chunk_sums = nullptr;
  uint8_t* chunk_raw = nullptr;
  uint8_t* chunk_flag = nullptr;
  int* chan_nflag = nullptr;
  double* mu = nullptr;
  double* sigma = nullptr;
  long long* S = nullptr;
  long long* V = nullptr;
  int* bint = nullptr;
  float* mu_hi = nullptr;
  float* mu_lo = nullptr;
  uint32_t* spec_bits = nullptr;
  int* spec_nflag = nullptr;
  double* spec_thr = nullptr;
  void* d_args = nullptr;     // device copy of this beam's dedispersion arguments
  long long* d_t0 = nullptr;  // device copy of t0_abs (read by the detection kernels)
  void* y = nullptr;          // staged series: FP32 for float data, 16-bit otherwise
  int64_t ypitch = 0;
  unsigned short* b16 = nullptr;
  double* bsum = nullptr;
  int* status = nullptr;
  void* D = nullptr;
  void* M = nullptr;          // median-filtered series (plans with median_width > 1)
  // clustering buffers (plans that cluster)
  int* cl_row_start = nullptr;
  int* cl_core = nullptr;
  int* cl_parent = nullptr;
  int* cl_root = nullptr;
  int* cl_rank = nullptr;
  int* cl_label = nullptr;
  int* cl_order = nullptr;
  int* cl_count = nullptr;
  int* cl_offset = nullptr;
  int* cl_cursor = nullptr;
  tp_cluster* clusters = nullptr;
  int* n_clusters = nullptr;
  int max_clusters = 0;
  float* pivot = nullptr;     // fitted bandpass buffers
  double* bfit = nullptr;
  uint8_t* fit_masked = nullptr;
  double* fit_work = nullptr;
  double* rmse = nullptr;
  void* post_part = nullptr;  // post-processing tile sums
  double* row_beta = nullptr;
  void* row_part = nullptr;
  double* row_mu = nullptr;
  double* row_sigma = nullptr;
  float* row_thr_f = nullptr;
  int* row_thr_i = nullptr;
  uint32_t* hit_bits = nullptr;
  uint32_t* blk_count = nullptr;
  uint32_t* blk_off = nullptr;
  tp_candidate* cand = nullptr;
  unsigned long long* n_total = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  // canary padding (tp_engine_set_canaries): each buffer's first byte and its
  // nominal size; kCanaryBytes of kCanaryByte sit before and after it
  std::vector<std::pair<unsigned char*, size_t>> canaries;
  int64_t dbg_y_bytes = -1;  // debug build: staged-series extent the checks use (tp_debug_limit_staged)
  // stream state
  int cur = 0;
  // the current window's first sample and row pitch (elements): win[cur], or
  // the caller's buffer after tp_push_inplace
  const void* xwin = nullptr;
  int64_t xpitch = 0;
  int64_t nsamp_win = 0;
  int64_t nout = 0;
  int64_t t0_abs = 0;
  int64_t pushed = 0;
  int64_t nblocks = 0;    // blocks pushed (running statistics alternate their state buffers)
  double* run_mu[2] = {nullptr, nullptr};   // running statistics (R15): state after even / odd blocks
  double* run_var[2] = {nullptr, nullptr};
  BeamState state = kEmpty;
  int ntt = 0;
  bool have_ext = false;
  // last arguments uploaded to d_args
  DedispArgs h_args{};
  int h_cta[2] = {0, 0};
  bool h_args_valid = false;
  // stage timing (tp_set_profiling)
  struct EventSet {
    cudaEvent_t ev[6];  // push start/end, rfi start, rfi end / dd start, dd end, detect end
  };
  std::vector<EventSet*> ev_pool;
  std::vector<EventSet*> ev_pending;
  EventSet* ev_cur = nullptr;
  double stage_ms[4] = {0, 0, 0, 0};
  int64_t stage_count = 0;
};

}  // namespace

struct tp_plan {
  tp_engine* e = nullptr;
  int nchan = 0, ndm = 0, max_delay = 0, dtype = 0;
  double f_lo = 0, bw = 0, t_samp = 0;
  std::vector<double> dm;
  tp_rfi_params rfi{};
  double nsigma = 5.0;
  int fit_order = -1;    // fitted bandpass (Sec. 2.2.1): polynomial order, -1 = off
  double run_alpha = 1.0;  // running statistics (R15): weight of the new block, 1 = per block
  double tau_mask = 5.0; // fitted bandpass: high-power channel masking threshold
  bool cluster = false;  // clustering of the detections (Sec. 2.3)
  tp_cluster_params cparams{};
  double* d_dmlist = nullptr;  // [ndm] DM values on the device (classification)
  int median_width = 1;  // post-processing (Sec. 2.2.3): median filter width, 1 = off
  int detrend = 0;       // post-processing: least-squares detrending
  int32_t* d_delay = nullptr;
  int32_t* d_delayT = nullptr;  // [nchan][ndm]
  std::vector<int32_t> h_delay;
  std::vector<DmTile> h_tiles;  // tiles of the selected shape
  DmTile* d_tiles = nullptr;
  int shape = 0;
  bool feasible[kNumShapes] = {};
  std::vector<DmTile> shape_tiles[kNumShapes];
  DmTile* d_shape_tiles[kNumShapes] = {};
  int users = 0;
  size_t bytes = 0;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  void* d_args = nullptr;  // the batch arguments the graph's launches read
};

struct tp_engine {
  int device = 0;
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  bool profiling = false;
  // batched dedispersion timing (tp_set_profiling, batches issued outside
  // graphs): event pairs around the grouped launches, harvested by
  // tp_get_batch_times
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> bev_pool, bev_pending;
  double batch_ms = 0.0;
  int64_t batch_count = 0;
  long long wait_tries = kDefaultWaitTries;  // see tp_engine_set_wait_limit
  // autotuner cache (tp_engine_set_tuning_cache): key -> (shape, ms per launch)
  std::string tune_path;
  std::map<std::string, std::pair<int, float>> tune_cache;
  bool canaries = false;  // beams opened from now on get canary padding
  int batch_grid = 0;  // batched dedispersion grid: 0 persistent, > 0 at most that many CTAs, < 0 one per item
  uint64_t launches = 0;
  void* d_batch = nullptr;  // batch arguments for launches outside graphs
  int* d_items = nullptr;   // work-item counters of the batched launches (one per kernel-shape group)
  std::vector<unsigned char> h_batch;
  std::map<std::string, GraphEntry> graphs;
  std::vector<tp_plan*> plans;
  std::vector<Beam*> beams;
  std::recursive_mutex mu;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    cudaGetDevice(&now);
    if (prev >= 0 && now != prev) cudaSetDevice(prev);
  }
};

int check_rfi(const tp_rfi_params& r) {
  if (r.chunk_width < 1) return set_error(TP_EINVAL, "chunk_width must be >= 1");
  if (!std::isfinite(r.tau_channel) || !std::isfinite(r.tau_spectrum))
    return set_error(TP_EINVAL, "thresholds must be finite");
  if (r.stats_mode != TP_STATS_BLOCK && r.stats_mode != TP_STATS_EXTERNAL)
    return set_error(TP_EINVAL, "unknown stats_mode %d", r.stats_mode);
  return TP_OK;
}

// Largest delay spread over channels between DM trials d0 and d1 (d0 <= d1;
// delays grow with DM for every channel).
int spread(const std::vector<int32_t>& delay, int nchan, int d0, int d1) {
  int s = 0;
  const int32_t* a = &delay[(size_t)d0 * nchan];
  const int32_t* b = &delay[(size_t)d1 * nchan];
  for (int c = 0; c < nchan; ++c) s = std::max(s, b[c] - a[c]);
  return s;
}

// Tiling for the dedispersion kernel with register shape `sh`: the shape is
// feasible when it stages the plan's sample size and every group of K
// consecutive trials spreads by at most OMAX - (16 / bytes per sample - 1)
// samples in every channel; tiles pack up to NCONS consecutive groups
// while the tile's delay spread stays within kMaxOverhang.
// Kernel shapes in order of preference when no autotuning has run: DM quads
// (paired-add forms first), then DM pairs, then direct loads, then register
// windows (the order of their launch times on a 1024-channel, 640-trial,
// 2^17-sample block).
constexpr int kShapePreference[kNumShapes] = {55, 53, 46, 56, 54, 52, 50, 51, 48, 49, 33, 44, 45,
                                              57, 58, 59, 60, 61, 62, 63, 64, 65, 66, 67, 47, 34, 42, 31, 30, 32, 35, 39, 43, 41, 40,
                                              27, 25, 26, 24, 28, 29, 22, 18, 19, 12, 13, 14, 15,
                                              16, 17, 23, 21, 20, 8, 10, 1, 2, 5, 0, 3, 6,
                                              4, 7, 9, 11, 36, 37, 38};

bool make_tiles(const std::vector<int32_t>& delay, int ndm, int nchan, int dtype, int sh,
                std::vector<DmTile>* tiles) {
  if (!format_ok(dtype, kShapes[sh].FMT)) return false;
  const int EB = staged_bytes_fmt(kShapes[sh].FMT);
  // per-beam buffers (partial sums, staging padding) are sized for tiles of
  // kMinTileT..kMaxTileT outputs
  if (shape_tile_t(sh) < kMinTileT || shape_tile_t(sh) > kMaxTileT) return false;
  const int K = kShapes[sh].K;
  const int residue = 16 / EB - 1;  // in-window offset of a 16-byte aligned copy
  if (kShapes[sh].ALGO == 2)
    // tiles start on even trials, so the pairs are (2i, 2i + 1): the second
    // trial's delay may exceed the first's by 0 .. OMAX in every channel
    for (int d0 = 0; d0 + 1 < ndm; d0 += 2) {
      const int32_t* a = &delay[(size_t)d0 * nchan];
      const int32_t* b = &delay[(size_t)(d0 + 1) * nchan];
      for (int c = 0; c < nchan; ++c)
        if (b[c] < a[c] || b[c] - a[c] > kShapes[sh].OMAX) return false;
    }
  if (kShapes[sh].ALGO >= 3)
    // quads (4i .. 4i + 3): in every channel the steps between consecutive
    // trials of a quad are m or m + 1 for one m in 0 .. OMAX
    for (int d0 = 0; d0 + 1 < ndm; d0 += K) {
      const int d1 = std::min(d0 + K, ndm) - 1;
      for (int c = 0; c < nchan; ++c) {
        int lo = 1 << 30, hi = -1;
        for (int d = d0 + 1; d <= d1; ++d) {
          const int e = delay[(size_t)d * nchan + c] - delay[(size_t)(d - 1) * nchan + c];
          lo = std::min(lo, e);
          hi = std::max(hi, e);
        }
        if (lo < 0 || hi - lo > 1 || lo > kShapes[sh].OMAX) return false;
      }
    }
  if (kShapes[sh].ALGO == 0)
    for (int d0 = 0; d0 < ndm; d0 += K) {
      const int d1 = std::min(d0 + K, ndm) - 1;
      if (spread(delay, nchan, d0, d1) + residue > kShapes[sh].OMAX) return false;
    }
  // the staging rows hold a tile's outputs plus at most kMaxOverhang samples
  // of delay spread, which a single group must respect too
  for (int d0 = 0; d0 < ndm; d0 += K)
    if (spread(delay, nchan, d0, std::min(d0 + K, ndm) - 1) > kMaxOverhang) return false;
  tiles->clear();
  int d0 = 0;
  while (d0 < ndm) {
    int ng = 1;
    while (ng < kShapes[sh].NCONS && d0 + ng * K < ndm) {
      const int d1 = std::min(d0 + (ng + 1) * K, ndm) - 1;
      if (spread(delay, nchan, d0, d1) > kMaxOverhang) break;
      ++ng;
    }
    const int nd = std::min(ng * K, ndm - d0);
    tiles->push_back(DmTile{d0, nd});
    d0 += nd;
  }
  return true;
}

Beam* get_beam(tp_engine* e, int id) {
  if (!e || id < 0 || id >= (int)e->beams.size()) return nullptr;
  return e->beams[id];
}

struct SizeItem {
  void** ptr;
  size_t bytes;    // allocated (multiple of 256)
  size_t nominal;  // what the buffer's layout needs
};

struct Sizes {
  size_t total = 0;
  std::vector<SizeItem> items;
};

// Canary padding around a beam's buffers (debugging aid, off by default):
// kCanaryBytes of kCanaryByte before each buffer and after its nominal size.
constexpr size_t kCanaryBytes = 256;
constexpr size_t kMaxGraphs = 64;  // cached batch graphs per engine
constexpr unsigned char kCanaryByte = 0xA5;

// Every device buffer of a beam, in one place (footprint and allocation).
void beam_layout(const tp_plan* p, int B, int cap, Beam* b, Sizes* out) {
  const size_t es = dtype_size(p->dtype);
  const int64_t nmax = (int64_t)p->max_delay + B;
  const int64_t pitch = (int64_t)round_up((size_t)nmax * es, 256) / (int64_t)es;
  const int W = p->rfi.chunk_width;
  const int nchunk = (int)((nmax + W - 1) / W);
  const int ntt = (int)((B + kMinTileT - 1) / kMinTileT);
  const int64_t ypitch = (int64_t)round_up((size_t)nmax + kMaxTileT + 64, 64);
  const int nblk = (int)((B + kDetectT - 1) / kDetectT);
  const int64_t hit_pitch = (B + 31) / 32;
  const int64_t dpitch = (int64_t)round_up((size_t)B, 64);
  b->pitch = pitch;
  b->nchunk_max = nchunk;
  b->ntt_max = ntt;
  b->nblk_max = nblk;
  b->hit_pitch = hit_pitch;
  b->dpitch = dpitch;
  b->ypitch = ypitch;
  const size_t nc = (size_t)p->nchan, nd = (size_t)p->ndm;
  auto add = [&](void** ptr, size_t bytes) {
    const size_t nominal = bytes;
    bytes = round_up(std::max<size_t>(bytes, 1), 256);
    out->items.push_back({ptr, bytes, nominal});
    out->total += bytes;
  };
  add(&b->win[0], nc * (size_t)pitch * es);
  add(&b->win[1], nc * (size_t)pitch * es);
  add(&b->chunk_sums, nc * (size_t)nchunk * 16);
  add((void**)&b->chunk_raw, nc * (size_t)nchunk);
  add((void**)&b->chunk_flag, nc * (size_t)nchunk);
  add((void**)&b->chan_nflag, nc * sizeof(int));
  add((void**)&b->mu, nc * 8);
  add((void**)&b->sigma, nc * 8);
  add((void**)&b->S, nc * 8);
  add((void**)&b->V, nc * 8);
  add((void**)&b->bint, nc * 4);
  add((void**)&b->mu_hi, nc * 4);
  add((void**)&b->mu_lo, nc * 4);
  add((void**)&b->spec_bits, (size_t)((nmax + 31) / 32) * 4);
  add((void**)&b->spec_nflag, 4);
  add((void**)&b->spec_thr, (size_t)nchunk * 8);
  add((void**)&b->pivot, nc * 4);
  add((void**)&b->bfit, nc * 8);
  add((void**)&b->fit_masked, nc);
  add((void**)&b->fit_work, nc * 16);
  add((void**)&b->rmse, 8);
  for (int i = 0; i < 2; ++i) {
    add((void**)&b->run_mu[i], nc * 8);
    add((void**)&b->run_var[i], nc * 8);
  }
  const size_t yb = (size_t)staged_bytes_alloc(p->dtype);
  add((void**)&b->y, nc * (size_t)ypitch * yb);
  add((void**)&b->b16, nc * 2);
  add((void**)&b->bsum, 8);
  add((void**)&b->status, 4);
  add(&b->d_args, sizeof(DedispArgs) + 16);
  add((void**)&b->d_t0, 8);
  add(&b->D, nd * (size_t)dpitch * 4);
  if (p->median_width > 1) add(&b->M, nd * (size_t)dpitch * 4);
  add(&b->post_part, nd * (size_t)nblk * 24);
  add((void**)&b->row_beta, nd * 8);
  add(&b->row_part, nd * (size_t)ntt * 16);
  add((void**)&b->row_mu, nd * 8);
  add((void**)&b->row_sigma, nd * 8);
  add((void**)&b->row_thr_f, nd * 4);
  add((void**)&b->row_thr_i, nd * 4);
  add((void**)&b->hit_bits, nd * (size_t)hit_pitch * 4);
  add((void**)&b->blk_count, nd * (size_t)nblk * 4);
  add((void**)&b->blk_off, nd * (size_t)nblk * 4);
  add((void**)&b->cand, (size_t)cap * sizeof(tp_candidate));
  if (p->cluster) {
    const int mc = cap < kMaxClusters ? cap : kMaxClusters;
    b->max_clusters = mc;
    add((void**)&b->cl_row_start, ((size_t)nd + 1) * 4);
    for (int** q : {&b->cl_core, &b->cl_parent, &b->cl_root, &b->cl_rank, &b->cl_label, &b->cl_order})
      add((void**)q, (size_t)cap * 4);
    add((void**)&b->cl_count, (size_t)mc * 4);
    add((void**)&b->cl_offset, ((size_t)mc + 1) * 4);
    add((void**)&b->cl_cursor, (size_t)mc * 4);
    add((void**)&b->clusters, (size_t)mc * sizeof(tp_cluster));
    add((void**)&b->n_clusters, 8);
  }
  add((void**)&b->n_total, 8);
}

void free_beam(Beam* b) {
  if (b->ev_cur) b->ev_pending.push_back(b->ev_cur);
  b->ev_cur = nullptr;
  for (auto* v : {&b->ev_pool, &b->ev_pending})
    for (Beam::EventSet* es : *v) {
      for (cudaEvent_t ev : es->ev) cudaEventDestroy(ev);
      delete es;
    }
  b->ev_pool.clear();
  b->ev_pending.clear();
  if (b->pf_stream) {
    cudaStreamSynchronize(b->pf_stream);  // a pending prefetch still reads the caller's buffer
    cudaStreamDestroy(b->pf_stream);
  }
  if (b->ev_win_free) cudaEventDestroy(b->ev_win_free);
  if (b->ev_pf) cudaEventDestroy(b->ev_pf);
  if (b->ev_detect) cudaEventDestroy(b->ev_detect);
  if (b->ev_pushed) cudaEventDestroy(b->ev_pushed);
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  b->canaries.clear();
}

cudaStream_t beam_stream(const tp_engine* e, const Beam* b) { return b->stream ? b->stream : e->stream; }

// Stage timing: an event set follows one block from push to detection.
void prof_harvest(Beam* b, bool wait) {
  size_t done = 0;
  for (; done < b->ev_pending.size(); ++done) {
    Beam::EventSet* es = b->ev_pending[done];
    if (wait) cudaEventSynchronize(es->ev[5]);
    else if (cudaEventQuery(es->ev[5]) != cudaSuccess) break;
    float ms[4] = {0, 0, 0, 0};
    cudaEventElapsedTime(&ms[0], es->ev[0], es->ev[1]);
    cudaEventElapsedTime(&ms[1], es->ev[2], es->ev[3]);
    cudaEventElapsedTime(&ms[2], es->ev[3], es->ev[4]);
    cudaEventElapsedTime(&ms[3], es->ev[4], es->ev[5]);
    for (int i = 0; i < 4; ++i) b->stage_ms[i] += ms[i];
    b->stage_count++;
    b->ev_pool.push_back(es);
  }
  b->ev_pending.erase(b->ev_pending.begin(), b->ev_pending.begin() + done);
  cudaGetLastError();
}

void prof_record(tp_engine* e, Beam* b, int which, cudaStream_t s) {
  if (!e->profiling) return;
  if (which == 0) {
    prof_harvest(b, false);
    if (b->ev_cur) {  // a block that never reached detection
      b->ev_pool.push_back(b->ev_cur);
      b->ev_cur = nullptr;
    }
    if (b->ev_pool.empty()) {
      auto* es = new Beam::EventSet();
      for (cudaEvent_t& ev : es->ev) cudaEventCreate(&ev);
      b->ev_pool.push_back(es);
    }
    b->ev_cur = b->ev_pool.back();
    b->ev_pool.pop_back();
  }
  if (!b->ev_cur) return;
  cudaEventRecord(b->ev_cur->ev[which], s);
  if (which == 5) {
    b->ev_pending.push_back(b->ev_cur);
    b->ev_cur = nullptr;
  }
}

RfiArgs rfi_args(const tp_plan* p, Beam* b) {
  RfiArgs a{};
  a.x = b->xwin;
  a.pitch = b->xpitch;
  a.nchan = p->nchan;
  a.nsamp = b->nsamp_win;
  a.W = p->rfi.chunk_width;
  a.nchunk = (int)((b->nsamp_win + a.W - 1) / a.W);
  a.dtype = p->dtype;
  a.stats_mode = p->rfi.stats_mode;
  a.enable_channel = p->rfi.enable_channel;
  a.enable_spectrum = p->rfi.enable_spectrum;
  a.dilate_channels = p->rfi.dilate_channels;
  a.tau_c = p->rfi.tau_channel;
  a.tau_s = p->rfi.tau_spectrum;
  a.mu = b->mu;
  a.sigma = b->sigma;
  a.S = b->S;
  a.V = b->V;
  a.bint = b->bint;
  a.mu_hi = b->mu_hi;
  a.mu_lo = b->mu_lo;
  a.b16 = b->b16;
  a.bsum = b->bsum;
  a.chunk_raw = b->chunk_raw;
  a.chunk_flag = b->chunk_flag;
  a.chan_nflag = b->chan_nflag;
  a.spec_bits = b->spec_bits;
  a.spec_nflag = b->spec_nflag;
  a.spec_thr = b->spec_thr;
  a.stage_f32 = (p->dtype == TP_F16 || p->dtype == TP_BF16) && kShapes[p->shape].FMT == 4;
  a.fit = p->fit_order >= 0 ? 1 : 0;
  a.fit_order = p->fit_order;
  a.tau_mask = p->tau_mask;
  a.pivot = b->pivot;
  a.bfit = b->bfit;
  a.fit_masked = b->fit_masked;
  a.fit_work = b->fit_work;
  a.rmse = b->rmse;
  a.run = p->run_alpha < 1.0 ? 1 : 0;
  a.run_alpha = p->run_alpha;
  // block n (1, 2, ...) folds the state of block n - 1 into buffer n % 2, so
  // that processing the same window again (tp_beam_rewind) repeats the same
  // update
  const int cur = (int)(b->nblocks & 1);
  a.run_first = b->nblocks <= 1 ? 1 : 0;
  a.run_prev_mu = b->run_mu[cur ^ 1];
  a.run_prev_var = b->run_var[cur ^ 1];
  a.run_mu = b->run_mu[cur];
  a.run_var = b->run_var[cur];
  a.status = b->status;
  a.x_elems = (int64_t)p->nchan * b->xpitch;
  a.y_elems = (int64_t)p->nchan * b->ypitch;
  return a;
}

DedispArgs dedisp_args(const tp_plan* p, Beam* b) {
  DedispArgs da{};
  da.y = b->y;
  da.ypitch = b->ypitch;
  da.bsum = b->bsum;
  da.nchan = p->nchan;
  da.nout = b->nout;
  da.dtype = p->dtype;
  da.delay = p->d_delay;
  da.delayT = p->d_delayT;
  da.dtpitch = p->ndm;
  da.ndm = p->ndm;
  da.tiles = p->d_tiles;
  da.ntiles = (int)p->h_tiles.size();
  da.shape = p->shape;
  da.ntt = (int)((b->nout + shape_tile_t(p->shape) - 1) / shape_tile_t(p->shape));
  da.D = b->D;
  da.dpitch = b->dpitch;
  da.row_part = b->row_part;
  da.status = b->status;
  da.y_bytes = (int64_t)p->nchan * b->ypitch * staged_bytes_alloc(p->dtype);
  if (b->dbg_y_bytes >= 0 && b->dbg_y_bytes < da.y_bytes) da.y_bytes = b->dbg_y_bytes;
  da.d_elems = (int64_t)p->ndm * b->dpitch;
  da.delayT_elems = (int64_t)p->nchan * p->ndm;
  return da;
}

// Launch the dedispersion kernel for one beam with shape `shape` (its args
// are re-uploaded only when they changed).
int launch_single(tp_engine* e, Beam* b, const DedispArgs& da, int shape, cudaStream_t s) {
  const int ctas = da.ntiles * da.ntt;
  if (da.ntt > b->ntt_max) return set_error(TP_EINVAL, "beam %d: %d time tiles exceed %d", b->id, da.ntt, b->ntt_max);
  if (!b->h_args_valid || std::memcmp(&b->h_args, &da, sizeof da) != 0 || b->h_cta[1] != ctas) {
    unsigned char buf[sizeof(DedispArgs) + 16];
    std::memcpy(buf, &da, sizeof da);
    const int cta[2] = {0, ctas};
    std::memcpy(buf + sizeof da, cta, sizeof cta);
    TP_CUDA_TRY(cudaMemcpyAsync(b->d_args, buf, sizeof buf, cudaMemcpyHostToDevice, s));
    b->h_args = da;
    b->h_cta[1] = ctas;
    b->h_args_valid = true;
  }
  BatchArgs ba{static_cast<const DedispArgs*>(b->d_args),
               reinterpret_cast<const int*>(static_cast<unsigned char*>(b->d_args) + sizeof(DedispArgs)), 1,
               nullptr, e->wait_tries};
  TP_CUDA_TRY(launch_dedisperse(shape, da.dtype, ba, ctas, s));
  e->launches += 1;
  return TP_OK;
}

int issue_rfi(tp_engine* e, Beam* b, cudaStream_t s) {
  const tp_plan* p = b->plan;
  if (b->state != kReady) return set_error(TP_ENOTREADY, "beam %d holds no new block", b->id);
  if (p->rfi.stats_mode == TP_STATS_EXTERNAL && !b->have_ext)
    return set_error(TP_ENOTREADY, "beam %d: external statistics not set", b->id);
  RfiArgs ra = rfi_args(p, b);
  int nk = 0;
  TP_CUDA_TRY(launch_rfi(ra, b->chunk_sums, b->y, b->ypitch, s, &nk));
  e->launches += nk;
  return TP_OK;
}

int issue_dedisperse(tp_engine* e, Beam* b) {
  const tp_plan* p = b->plan;
  cudaStream_t s = beam_stream(e, b);
  if (b->state == kReady) prof_record(e, b, 2, s);
  int rc = issue_rfi(e, b, s);
  if (rc) return rc;
  prof_record(e, b, 3, s);
  DedispArgs da = dedisp_args(p, b);
  b->ntt = da.ntt;
  rc = launch_single(e, b, da, p->shape, s);
  if (rc) return rc;
  prof_record(e, b, 4, s);
  b->state = kDedispersed;
  return TP_OK;
}

int issue_detect(tp_engine* e, Beam* b, cudaStream_t s) {
  const tp_plan* p = b->plan;
  if (b->state != kDedispersed) return set_error(TP_ENOTREADY, "beam %d is not dedispersed", b->id);
  DetectArgs a{};
  a.D = b->D;
  a.dpitch = b->dpitch;
  a.ndm = p->ndm;
  a.nout = b->nout;
  a.is_int = p->dtype == TP_U8;
  a.row_part = b->row_part;
  a.ntt = b->ntt;
  a.nsigma = p->nsigma;
  a.beam = b->id;
  a.t0_abs = b->d_t0;
  a.row_mu = b->row_mu;
  a.row_sigma = b->row_sigma;
  a.row_thr_f = b->row_thr_f;
  a.row_thr_i = b->row_thr_i;
  a.hit_bits = b->hit_bits;
  a.hit_pitch = (b->nout + 31) / 32;
  a.blk_count = b->blk_count;
  a.blk_off = b->blk_off;
  a.nblk_t = (int)((b->nout + kDetectT - 1) / kDetectT);
  a.cand = b->cand;
  a.cap = b->cap;
  a.n_total = b->n_total;
  a.median_width = p->median_width;
  a.detrend = p->detrend;
  a.M = b->M;
  a.post_part = b->post_part;
  a.row_beta = b->row_beta;
  a.status = b->status;
  a.d_elems = (int64_t)p->ndm * b->dpitch;
  a.hit_elems = (int64_t)p->ndm * b->hit_pitch;
  TP_CUDA_TRY(launch_detect(a, s));
  e->launches += (p->median_width > 1 || p->detrend) ? 5 : 4;
  if (p->cluster) {
    ClusterArgs c{};
    c.cand = b->cand;
    c.n_total = b->n_total;
    c.cap = b->cap;
    c.ndm = p->ndm;
    c.dm = p->d_dmlist;
    c.t_samp = p->t_samp;
    c.bw_mhz = std::fabs(p->bw);
    c.f_ghz = (p->f_lo + p->bw / 2.0) / 1e3;
    c.t_eps = p->cparams.t_eps;
    c.dm_eps = p->cparams.dm_eps;
    c.snr_eps = (float)p->cparams.snr_eps;
    c.min_pts = p->cparams.min_pts;
    c.smooth = p->cparams.smooth;
    c.rmse_max = p->cparams.rmse_max;
    c.dm_min = p->cparams.dm_min;
    c.row_start = b->cl_row_start;
    c.core = b->cl_core;
    c.parent = b->cl_parent;
    c.root = b->cl_root;
    c.rank = b->cl_rank;
    c.label = b->cl_label;
    c.order = b->cl_order;
    c.max_clusters = b->max_clusters;
    c.cl_count = b->cl_count;
    c.cl_offset = b->cl_offset;
    c.cl_cursor = b->cl_cursor;
    c.clusters = b->clusters;
    c.n_clusters = b->n_clusters;
    c.truncated = b->n_clusters + 1;
    TP_CUDA_TRY(launch_cluster(c, s));
    e->launches += 9;
  }
  prof_record(e, b, 5, s);
  TP_CUDA_TRY(cudaEventRecord(b->ev_detect, s));
  b->state = kDetected;
  return TP_OK;
}

// ---- batches: every beam holding a new block, one dedispersion launch per
// (kernel shape, sample format) group, all on the engine stream.
struct BatchPlan {
  std::vector<Beam*> beams;                         // in launch order
  std::vector<std::pair<int, int>> groups;          // (first index, count)
  std::vector<DedispArgs> args;                     // per beam
  std::vector<int> cta;                             // per group: count + 1 starts, concatenated
  std::string key;
};

BatchPlan plan_batch(tp_engine* e) {
  BatchPlan bp;
  std::vector<Beam*> ready;
  for (Beam* b : e->beams)
    if (b && b->state == kReady) ready.push_back(b);
  std::stable_sort(ready.begin(), ready.end(), [](const Beam* x, const Beam* y) {
    const int mx = x->plan->dtype == TP_BF16, my = y->plan->dtype == TP_BF16;
    return x->plan->shape != y->plan->shape ? x->plan->shape < y->plan->shape : mx < my;
  });
  char tmp[160];
  for (size_t i = 0; i < ready.size(); ++i) {
    Beam* b = ready[i];
    const bool start = i == 0 || ready[i - 1]->plan->shape != b->plan->shape ||
                       (ready[i - 1]->plan->dtype == TP_BF16) != (b->plan->dtype == TP_BF16);
    if (start) bp.groups.push_back({(int)i, 0});
    bp.groups.back().second++;
    bp.beams.push_back(b);
    DedispArgs da = dedisp_args(b->plan, b);
    if (da.ntt > b->ntt_max) {
      bp.beams.clear();
      bp.key = "error";
      return bp;
    }
    bp.args.push_back(da);
    snprintf(tmp, sizeof tmp, "%d:%p:%lld:%lld:%d:%d;", b->id, b->xwin, (long long)b->xpitch,
             (long long)b->nout, b->plan->shape, (int)b->plan->h_tiles.size());
    bp.key += tmp;
  }
  for (auto& g : bp.groups) {
    int acc = 0;
    for (int k = 0; k < g.second; ++k) {
      bp.cta.push_back(acc);
      const DedispArgs& a = bp.args[g.first + k];
      acc += a.ntiles * a.ntt;
    }
    bp.cta.push_back(acc);
  }
  return bp;
}

size_t batch_bytes(const BatchPlan& bp) { return bp.args.size() * sizeof(DedispArgs) + bp.cta.size() * 4 + 16; }

// Issue RFI + batched dedispersion + detection for a planned batch; batch
// arguments at `d_args` (device) must already hold the plan's arguments.
// The engine stream waits for the pushes of beams that have their own stream.
int wait_pushes(tp_engine* e, const BatchPlan& bp) {
  for (Beam* b : bp.beams)
    if (b->stream && b->stream != e->stream) TP_CUDA_TRY(cudaStreamWaitEvent(e->stream, b->ev_pushed, 0));
  return TP_OK;
}

int issue_batch(tp_engine* e, BatchPlan& bp, void* d_args, bool detect) {
  cudaStream_t s = e->stream;
  for (Beam* b : bp.beams) {
    int rc = issue_rfi(e, b, s);
    if (rc) return rc;
  }
  const DedispArgs* dargs = static_cast<const DedispArgs*>(d_args);
  const int* dcta = reinterpret_cast<const int*>(static_cast<unsigned char*>(d_args) +
                                                 bp.args.size() * sizeof(DedispArgs));
  int coff = 0;
  // one work-item counter per kernel-shape group of the batch
  if (bp.groups.size() > kMaxBatchGroups) return set_error(TP_EINVAL, "more than %d kernel-shape groups", kMaxBatchGroups);
  TP_CUDA_TRY(cudaMemsetAsync(e->d_items, 0, sizeof(int) * bp.groups.size(), s));
  int gi = 0;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (e->profiling) {  // never set while a graph is captured
    if (e->bev_pool.empty()) {
      TP_CUDA_TRY(cudaEventCreate(&ev.first));
      TP_CUDA_TRY(cudaEventCreate(&ev.second));
    } else {
      ev = e->bev_pool.back();
      e->bev_pool.pop_back();
    }
    TP_CUDA_TRY(cudaEventRecord(ev.first, s));
  }
  for (auto& g : bp.groups) {
    BatchArgs ba{dargs + g.first, dcta + coff, g.second, e->d_items + gi++, e->wait_tries};
    const int ctas = bp.cta[coff + g.second];
    const Beam* b0 = bp.beams[g.first];
    TP_CUDA_TRY(launch_dedisperse(b0->plan->shape, b0->plan->dtype, ba, ctas, s, e->batch_grid));
    e->launches += 1;
    coff += g.second + 1;
  }
  if (ev.first) {
    TP_CUDA_TRY(cudaEventRecord(ev.second, s));
    e->bev_pending.push_back(ev);
  }
  for (size_t i = 0; i < bp.beams.size(); ++i) {
    bp.beams[i]->ntt = bp.args[i].ntt;
    bp.beams[i]->state = kDedispersed;
  }
  if (detect)
    for (Beam* b : bp.beams) {
      int rc = issue_detect(e, b, s);
      if (rc) return rc;
    }
  return TP_OK;
}

void pack_batch(const BatchPlan& bp, std::vector<unsigned char>* out) {
  out->resize(batch_bytes(bp));
  std::memcpy(out->data(), bp.args.data(), bp.args.size() * sizeof(DedispArgs));
  std::memcpy(out->data() + bp.args.size() * sizeof(DedispArgs), bp.cta.data(), bp.cta.size() * 4);
}

}  // namespace

namespace tp {
const char* last_error_cstr();
}

extern "C" {

void tp_rfi_defaults(tp_rfi_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->enable_channel = 1;
  p->enable_spectrum = 1;
  p->chunk_width = 256;
  p->dilate_channels = 0;
  p->tau_channel = 5.0;
  p->tau_spectrum = 6.0;
  p->stats_mode = TP_STATS_BLOCK;
}

int tp_version(void) { return 200; }

const char* tp_last_error_string(void) { return tp::last_error_cstr(); }

int tp_engine_create(int device, size_t hbm_budget_bytes, void* cuda_stream, tp_engine** out) {
  TP_NVTX_RANGE();
  if (!out) return set_error(TP_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  TP_CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return set_error(TP_EINVAL, "device %d of %d", device, n);
  DeviceGuard g(device);
  size_t free_b = 0, total_b = 0;
  TP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  tp_engine* e = new (std::nothrow) tp_engine();
  if (!e) return set_error(TP_ENOMEM, "engine allocation");
  if (cudaMalloc(&e->d_batch, kBatchBytes) != cudaSuccess ||
      cudaMalloc(&e->d_items, sizeof(int) * kMaxBatchGroups) != cudaSuccess) {
    cudaFree(e->d_batch);
    delete e;
    return set_error(TP_ENOMEM, "engine batch arguments");
  }
  e->device = device;
  e->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  e->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = e;
  return TP_OK;
}

int tp_engine_destroy(tp_engine* e) {
  TP_NVTX_RANGE();
  if (!e) return TP_OK;
  {
    std::lock_guard<std::recursive_mutex> lk(e->mu);
    DeviceGuard g(e->device);
    cudaStreamSynchronize(e->stream);
    for (Beam* b : e->beams)
      if (b) {
        cudaStreamSynchronize(beam_stream(e, b));
        free_beam(b);
        delete b;
      }
    e->beams.clear();
    for (tp_plan* p : e->plans) {
      cudaFree(p->d_dmlist);
      cudaFree(p->d_delay);
      cudaFree(p->d_delayT);
      for (DmTile* t : p->d_shape_tiles) cudaFree(t);
      delete p;
    }
    e->plans.clear();
    for (auto& kv : e->graphs) {
      cudaGraphExecDestroy(kv.second.exec);
      cudaFree(kv.second.d_args);
    }
    e->graphs.clear();
    for (auto* v : {&e->bev_pool, &e->bev_pending})
      for (auto& ev : *v) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
      }
    cudaFree(e->d_batch);
    cudaFree(e->d_items);
  }
  delete e;
  return TP_OK;
}

int tp_sync(tp_engine* e) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  TP_CUDA_TRY(cudaStreamSynchronize(e->stream));
  for (Beam* b : e->beams)
    if (b && b->stream) TP_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return TP_OK;
}

int tp_engine_stream(const tp_engine* e, void** stream) {
  if (!e || !stream) return set_error(TP_EINVAL, "engine or stream is NULL");
  *stream = e->stream;
  return TP_OK;
}

int tp_engine_memory(const tp_engine* e, size_t* used, size_t* budget) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  if (used) *used = e->used;
  if (budget) *budget = e->budget;
  return TP_OK;
}

int tp_create_plan(tp_engine* e, int nchan, double f_lo_mhz, double bw_mhz, double t_samp_s,
                   const double* dm_list, int ndm, int dtype, const tp_rfi_params* rfi,
                   double nsigma, tp_plan** out) {
  TP_NVTX_RANGE();
  if (!e || !out) return set_error(TP_EINVAL, "engine or out is NULL");
  *out = nullptr;
  if (nchan <= 0 || ndm <= 0) return set_error(TP_EINVAL, "nchan %d / ndm %d must be > 0", nchan, ndm);
  if (nchan > 65535) return set_error(TP_EINVAL, "nchan %d: at most 65535 channels", nchan);
  if (!(t_samp_s > 0.0) || !std::isfinite(t_samp_s)) return set_error(TP_EINVAL, "t_samp must be > 0");
  if (!std::isfinite(f_lo_mhz) || !std::isfinite(bw_mhz) || bw_mhz == 0.0)
    return set_error(TP_EINVAL, "f_lo / bw invalid");
  if (dtype_size(dtype) == 0) return set_error(TP_EINVAL, "unknown dtype %d", dtype);
  if (!dm_list) return set_error(TP_EINVAL, "dm_list is NULL");
  if (!std::isfinite(nsigma)) return set_error(TP_EINVAL, "nsigma must be finite");
  for (int d = 0; d < ndm; ++d) {
    if (!std::isfinite(dm_list[d]) || dm_list[d] < 0.0)
      return set_error(TP_EINVAL, "DM %d is negative or not finite", d);
    if (d > 0 && dm_list[d] < dm_list[d - 1]) return set_error(TP_EINVAL, "DM list must be non-decreasing");
  }
  const double df = bw_mhz / nchan;
  const double fa = f_lo_mhz + 0.5 * df, fb = f_lo_mhz + ((double)nchan - 0.5) * df;
  if (!(fa > 0.0) || !(fb > 0.0)) return set_error(TP_EINVAL, "channel frequencies must be > 0");
  tp_rfi_params r;
  if (rfi) r = *rfi;
  else tp_rfi_defaults(&r);
  int rc = check_rfi(r);
  if (rc) return rc;

  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  tp_plan* p = new tp_plan();
  p->e = e;
  p->nchan = nchan;
  p->ndm = ndm;
  p->dtype = dtype;
  p->f_lo = f_lo_mhz;
  p->bw = bw_mhz;
  p->t_samp = t_samp_s;
  p->dm.assign(dm_list, dm_list + ndm);
  p->rfi = r;
  p->nsigma = nsigma;
  const size_t n = (size_t)nchan * ndm;
  double* d_dm = nullptr;
  int* d_err = nullptr;
  auto fail = [&](int code) {
    cudaFree(d_dm);
    cudaFree(d_err);
    cudaFree(p->d_dmlist);
    cudaFree(p->d_delay);
    cudaFree(p->d_delayT);
    for (DmTile* t : p->d_shape_tiles) cudaFree(t);
    delete p;
    return code;
  };
  cudaError_t ce;
  if ((ce = cudaMalloc(&p->d_delay, n * 4)) != cudaSuccess) return fail(cuda_error(ce, "cudaMalloc(delay)"));
  if ((ce = cudaMalloc(&d_dm, ndm * 8)) != cudaSuccess) return fail(cuda_error(ce, "cudaMalloc(dm)"));
  if ((ce = cudaMalloc(&d_err, 4)) != cudaSuccess) return fail(cuda_error(ce, "cudaMalloc(err)"));
  if ((ce = cudaMemcpyAsync(d_dm, dm_list, ndm * 8, cudaMemcpyHostToDevice, e->stream)) != cudaSuccess)
    return fail(cuda_error(ce, "copy dm"));
  if ((ce = cudaMemsetAsync(d_err, 0, 4, e->stream)) != cudaSuccess) return fail(cuda_error(ce, "memset"));
  if ((ce = launch_delay_table(nchan, f_lo_mhz, bw_mhz, t_samp_s, d_dm, ndm, p->d_delay, d_err, e->stream)) !=
      cudaSuccess)
    return fail(cuda_error(ce, "delay table kernel"));
  e->launches += 1;
  p->h_delay.resize(n);
  int herr = 0;
  if ((ce = cudaMemcpyAsync(p->h_delay.data(), p->d_delay, n * 4, cudaMemcpyDeviceToHost, e->stream)) !=
      cudaSuccess)
    return fail(cuda_error(ce, "copy delay"));
  if ((ce = cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, e->stream)) != cudaSuccess)
    return fail(cuda_error(ce, "copy err"));
  if ((ce = cudaStreamSynchronize(e->stream)) != cudaSuccess) return fail(cuda_error(ce, "sync"));
  p->d_dmlist = d_dm;  // kept for the classification of clusters
  d_dm = nullptr;
  cudaFree(d_err);
  d_err = nullptr;
  if (herr) return fail(set_error(TP_EINVAL, "a delay exceeds 2^31 - 1 samples"));
  int dmax = 0;
  for (int32_t v : p->h_delay) dmax = std::max(dmax, (int)v);
  p->max_delay = dmax;
  p->shape = -1;
  size_t tb = 0;
  for (int sh = 0; sh < kNumShapes; ++sh) {
    p->feasible[sh] = make_tiles(p->h_delay, ndm, nchan, dtype, sh, &p->shape_tiles[sh]);
    if (!p->feasible[sh]) continue;
    const size_t bts = p->shape_tiles[sh].size() * sizeof(DmTile);
    if ((ce = cudaMalloc(&p->d_shape_tiles[sh], bts)) != cudaSuccess) return fail(cuda_error(ce, "cudaMalloc(tiles)"));
    if ((ce = cudaMemcpy(p->d_shape_tiles[sh], p->shape_tiles[sh].data(), bts, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return fail(cuda_error(ce, "copy tiles"));
    tb += bts;
  }
  // default shape (until tp_autotune or tp_plan_set_shape): the first
  // feasible one in an order of measured speed on the 1024-channel band
  for (int sh : kShapePreference)
    if (p->feasible[sh]) {
      p->shape = sh;
      break;
    }
  if (p->shape < 0) return fail(set_error(TP_EINVAL, "no kernel shape fits this DM list"));
  p->h_tiles = p->shape_tiles[p->shape];
  p->d_tiles = p->d_shape_tiles[p->shape];
  {
    std::vector<int32_t> tr(n);
    for (int d = 0; d < ndm; ++d)
      for (int c = 0; c < nchan; ++c) tr[(size_t)c * ndm + d] = p->h_delay[(size_t)d * nchan + c];
    if ((ce = cudaMalloc(&p->d_delayT, n * 4)) != cudaSuccess) return fail(cuda_error(ce, "cudaMalloc(delayT)"));
    if ((ce = cudaMemcpy(p->d_delayT, tr.data(), n * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(cuda_error(ce, "copy delayT"));
  }
  p->bytes = 2 * n * 4 + tb;
  e->used += p->bytes;
  e->plans.push_back(p);
  *out = p;
  return TP_OK;
}

int tp_plan_destroy(tp_plan* p) {
  TP_NVTX_RANGE();
  if (!p) return TP_OK;
  tp_engine* e = p->e;
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  if (p->users > 0) return set_error(TP_EBUSY, "plan is used by %d open beams", p->users);
  DeviceGuard g(e->device);
  cudaStreamSynchronize(e->stream);
  cudaFree(p->d_dmlist);
  cudaFree(p->d_delay);
  cudaFree(p->d_delayT);
  for (DmTile* t : p->d_shape_tiles) cudaFree(t);
  e->used -= p->bytes;
  e->plans.erase(std::remove(e->plans.begin(), e->plans.end(), p), e->plans.end());
  delete p;
  return TP_OK;
}

int tp_plan_info(const tp_plan* p, int* nchan, int* ndm, int* max_delay, int* dtype) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  if (nchan) *nchan = p->nchan;
  if (ndm) *ndm = p->ndm;
  if (max_delay) *max_delay = p->max_delay;
  if (dtype) *dtype = p->dtype;
  return TP_OK;
}

int tp_get_delay_table(const tp_plan* p, int32_t* out, size_t count) {
  if (!p || !out) return set_error(TP_EINVAL, "plan or out is NULL");
  if (count < p->h_delay.size()) return set_error(TP_EINVAL, "buffer holds %zu of %zu", count, p->h_delay.size());
  std::memcpy(out, p->h_delay.data(), p->h_delay.size() * 4);
  return TP_OK;
}

int tp_beam_footprint(const tp_plan* p, int block_nsamp, int cand_capacity, size_t* bytes) {
  if (!p || !bytes) return set_error(TP_EINVAL, "plan or bytes is NULL");
  if (block_nsamp <= p->max_delay)
    return set_error(TP_EINVAL, "block_nsamp %d must exceed the largest delay %d", block_nsamp, p->max_delay);
  if (cand_capacity < 1) return set_error(TP_EINVAL, "cand_capacity must be >= 1");
  Beam tmp;
  Sizes sz;
  beam_layout(p, block_nsamp, cand_capacity, &tmp, &sz);
  *bytes = sz.total;
  return TP_OK;
}

int tp_beam_open(tp_engine* e, const tp_plan* p, int block_nsamp, int cand_capacity, int* beam_id) {
  TP_NVTX_RANGE();
  if (!e || !p || !beam_id) return set_error(TP_EINVAL, "engine, plan or beam_id is NULL");
  if (p->e != e) return set_error(TP_EINVAL, "plan belongs to another engine");
  size_t need = 0;
  int rc = tp_beam_footprint(p, block_nsamp, cand_capacity, &need);
  if (rc) return rc;
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  if (e->used + need > e->budget)
    return set_error(TP_EADMIT, "beam needs %zu bytes, %zu of %zu in use", need, e->used, e->budget);
  DeviceGuard g(e->device);
  Beam* b = new Beam();
  b->e = e;
  b->plan = p;
  b->B = block_nsamp;
  b->cap = cand_capacity;
  Sizes sz;
  beam_layout(p, block_nsamp, cand_capacity, b, &sz);
  for (auto& it : sz.items) {
    void* ptr = nullptr;
    const size_t pad = e->canaries ? kCanaryBytes : 0;
    const size_t bytes = it.bytes + 2 * pad;
    cudaError_t ce = cudaMalloc(&ptr, bytes);
    if (ce == cudaSuccess) b->allocs.push_back(ptr);
    if (ce == cudaSuccess && pad) {
      unsigned char* base = static_cast<unsigned char*>(ptr);
      ce = cudaMemset(base, kCanaryByte, pad);
      if (ce == cudaSuccess) ce = cudaMemset(base + pad + it.nominal, kCanaryByte, bytes - pad - it.nominal);
      b->canaries.push_back({base + pad, it.nominal});
    }
    if (ce != cudaSuccess) {
      cudaGetLastError();
      free_beam(b);
      delete b;
      return set_error(TP_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(ce));
    }
    *it.ptr = static_cast<unsigned char*>(ptr) + pad;
  }
  cudaError_t ce = cudaMemset(b->y, 0, (size_t)p->nchan * b->ypitch * (size_t)staged_bytes_alloc(p->dtype));
  if (ce == cudaSuccess) ce = cudaMemset(b->status, 0, 4);
  if (ce != cudaSuccess) {
    free_beam(b);
    delete b;
    return cuda_error(ce, "cudaMemset");
  }
  ce = cudaEventCreateWithFlags(&b->ev_detect, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_pushed, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_win_free, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ev_pf, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    free_beam(b);
    delete b;
    return cuda_error(ce, "cudaEventCreate");
  }
  b->bytes = sz.total;
  int id = -1;
  for (int i = 0; i < (int)e->beams.size(); ++i)
    if (!e->beams[i]) {
      id = i;
      break;
    }
  if (id < 0) {
    id = (int)e->beams.size();
    e->beams.push_back(nullptr);
  }
  b->id = id;
  e->beams[id] = b;
  e->used += b->bytes;
  const_cast<tp_plan*>(p)->users++;
  *beam_id = id;
  return TP_OK;
}

int tp_beam_close(tp_engine* e, int beam) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  DeviceGuard g(e->device);
  cudaStreamSynchronize(beam_stream(e, b));
  const_cast<tp_plan*>(b->plan)->users--;
  e->used -= b->bytes;
  free_beam(b);
  e->beams[beam] = nullptr;
  delete b;
  return TP_OK;
}

int tp_beam_rewind(tp_engine* e, int beam) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->nsamp_win == 0) return set_error(TP_ENOTREADY, "beam %d holds no block", beam);
  b->state = kReady;
  return TP_OK;
}

int tp_beam_set_stream(tp_engine* e, int beam, void* cuda_stream) {
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  return TP_OK;
}

int tp_beam_set_bandpass(tp_engine* e, int beam, const double* mu, const double* sigma, int nchan) {
  TP_NVTX_RANGE();
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  const tp_plan* p = b->plan;
  if (p->rfi.stats_mode != TP_STATS_EXTERNAL)
    return set_error(TP_EINVAL, "plan does not use external statistics");
  if (!mu || !sigma || nchan != p->nchan) return set_error(TP_EINVAL, "need %d mu and sigma values", p->nchan);
  for (int c = 0; c < nchan; ++c)
    if (!std::isfinite(mu[c]) || !std::isfinite(sigma[c]) || sigma[c] < 0.0)
      return set_error(TP_EINVAL, "channel %d: mu/sigma invalid", c);
  std::vector<float> hi(nchan), lo(nchan);
  std::vector<int> bi(nchan);
  std::vector<unsigned short> bh(nchan);
  for (int c = 0; c < nchan; ++c) {
    hi[c] = (float)mu[c];
    lo[c] = (float)(mu[c] - (double)hi[c]);
    bi[c] = (int)std::floor(mu[c] + 0.5);
    bh[c] = p->dtype == TP_F16 || p->dtype == TP_BF16 ? storage_bits_host(p->dtype, mu[c]) : 0;
  }
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  TP_CUDA_TRY(cudaMemcpyAsync(b->mu, mu, nchan * 8, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(b->sigma, sigma, nchan * 8, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(b->mu_hi, hi.data(), nchan * 4, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(b->mu_lo, lo.data(), nchan * 4, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(b->bint, bi.data(), nchan * 4, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(b->b16, bh.data(), nchan * 2, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
  b->have_ext = true;
  return TP_OK;
}

namespace {

// Checks shared by the pushes: the size, the beam's state and the first
// block's length.
int check_push(const Beam* b, int nsamp, int beam) {
  if (nsamp < 1 || nsamp > b->B) return set_error(TP_EINVAL, "nsamp %d not in [1, %d]", nsamp, b->B);
  if (b->state == kReady || b->state == kDedispersed)
    return set_error(TP_EBUSY, "beam %d: previous block not yet through detection", beam);
  if (b->pushed == 0 && nsamp <= b->plan->max_delay)
    return set_error(TP_EINVAL, "first block (%d samples) must exceed the largest delay %lld", nsamp,
                     (long long)b->plan->max_delay);
  return TP_OK;
}

// Assembles the next window on stream s: the overlap tail of the current
// window, then (unless the new samples are already in place) the new block
// from `buf` (row pitch `spitch` bytes); then publishes the block (t0, events,
// state).  inplace_pitch > 0 (tp_push_inplace): from the stream's second
// block on, the window is the caller's buffer itself (row pitch inplace_pitch
// elements), which receives only the tail in its first max_delay columns.
int assemble_window(tp_engine* e, Beam* b, cudaStream_t s, const void* buf, size_t spitch, int nsamp,
                    int buf_is_device, int64_t inplace_pitch = 0) {
  const tp_plan* p = b->plan;
  const int64_t dmax = p->max_delay;
  const size_t es = dtype_size(p->dtype);
  const cudaMemcpyKind kind = buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t dpitch = (size_t)b->pitch * es;
  const size_t rowb = (size_t)nsamp * es;
  // on its own stream, a push must not overwrite the window, t0 or buffers
  // while the beam's previous batch may still run on the engine stream
  if (s != e->stream && b->pushed > 0) TP_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_detect, 0));
  prof_record(e, b, 0, s);
  int nk = 0;  // copy kernels launched
  if (b->pushed == 0) {
    b->cur = 0;
    if (buf && buf_is_device)
      TP_CUDA_TRY(copy_rows(b->win[0], dpitch, buf, spitch, rowb, p->nchan, s, &nk));
    else if (buf)
      TP_CUDA_TRY(cudaMemcpy2DAsync(b->win[0], dpitch, buf, spitch, rowb, p->nchan, kind, s));
    b->xwin = b->win[0];
    b->xpitch = b->pitch;
    b->nsamp_win = nsamp;
    b->nout = nsamp - dmax;
    b->t0_abs = 0;
  } else {
    const char* tail = static_cast<const char*>(b->xwin) + (size_t)(b->nsamp_win - dmax) * es;
    const size_t tpitch = (size_t)b->xpitch * es;
    if (inplace_pitch > 0) {
      char* dst = static_cast<char*>(const_cast<void*>(buf));
      if (dmax > 0)
        TP_CUDA_TRY(copy_rows(dst, (size_t)inplace_pitch * es, tail, tpitch, (size_t)dmax * es, p->nchan, s, &nk));
      b->xwin = buf;
      b->xpitch = inplace_pitch;
    } else {
      const int nxt = b->cur ^ 1;
      char* dst = static_cast<char*>(b->win[nxt]);
      if (dmax > 0) TP_CUDA_TRY(copy_rows(dst, dpitch, tail, tpitch, (size_t)dmax * es, p->nchan, s, &nk));
      if (buf && buf_is_device)
        TP_CUDA_TRY(copy_rows(dst + (size_t)dmax * es, dpitch, buf, spitch, rowb, p->nchan, s, &nk));
      else if (buf)
        TP_CUDA_TRY(cudaMemcpy2DAsync(dst + (size_t)dmax * es, dpitch, buf, spitch, rowb, p->nchan, kind, s));
      b->cur = nxt;
      b->xwin = b->win[nxt];
      b->xpitch = b->pitch;
    }
    b->nsamp_win = dmax + nsamp;
    b->nout = nsamp;
    b->t0_abs = b->pushed - dmax;
  }
  // the other window is free once the tail has been copied out of it (and,
  // earlier on this stream, the previous block's kernels have read it)
  TP_CUDA_TRY(cudaEventRecord(b->ev_win_free, s));
  e->launches += (uint64_t)nk;
  TP_CUDA_TRY(cudaMemcpyAsync(b->d_t0, &b->t0_abs, 8, cudaMemcpyHostToDevice, s));
  TP_CUDA_TRY(cudaEventRecord(b->ev_pushed, s));
  prof_record(e, b, 1, s);
  b->pushed += nsamp;
  b->nblocks += 1;
  b->state = kReady;
  return TP_OK;
}

}  // namespace

int tp_push_block(tp_engine* e, int beam, const void* buf, int nsamp, int buf_is_device) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (!buf) return set_error(TP_EINVAL, "buf is NULL");
  if (b->pf_pending) return set_error(TP_EBUSY, "beam %d has a prefetched block to push first", beam);
  const int rc = check_push(b, nsamp, beam);
  if (rc != TP_OK) return rc;
  DeviceGuard g(e->device);
  return assemble_window(e, b, beam_stream(e, b), buf, (size_t)nsamp * dtype_size(b->plan->dtype), nsamp,
                         buf_is_device);
}

int tp_push_inplace(tp_engine* e, int beam, void* buf, int64_t pitch, int nsamp) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (!buf) return set_error(TP_EINVAL, "buf is NULL");
  if (b->pf_pending) return set_error(TP_EBUSY, "beam %d has a prefetched block to push first", beam);
  const int rc = check_push(b, nsamp, beam);
  if (rc != TP_OK) return rc;
  const tp_plan* p = b->plan;
  const size_t es = dtype_size(p->dtype);
  if (pitch < p->max_delay + (int64_t)nsamp)
    return set_error(TP_EINVAL, "pitch %lld below max_delay + nsamp = %lld", (long long)pitch,
                     (long long)(p->max_delay + nsamp));
  // the kernels load the window in 16-byte units
  if ((reinterpret_cast<uintptr_t>(buf) | (uintptr_t)((size_t)pitch * es)) % 16 != 0)
    return set_error(TP_EINVAL, "buf and the row pitch (%lld elements) must be 16-byte multiples", (long long)pitch);
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, buf) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
      attr.device != e->device) {
    cudaGetLastError();
    return set_error(TP_EINVAL, "buf is not device memory of the engine's device");
  }
  // the previous block's samples (the tail to copy) live in its own buffer
  if (b->pushed > 0 && buf == b->xwin)
    return set_error(TP_EINVAL, "buf holds the previous block: alternate at least two buffers");
  DeviceGuard g(e->device);
  const char* block = static_cast<const char*>(buf) + (size_t)p->max_delay * es;
  if (b->pushed == 0)  // the stream's first block: copied into the engine's window
    return assemble_window(e, b, beam_stream(e, b), block, (size_t)pitch * es, nsamp, 1);
  return assemble_window(e, b, beam_stream(e, b), buf, (size_t)pitch * es, nsamp, 1, pitch);
}

int tp_prefetch_block(tp_engine* e, int beam, const void* host_buf, int nsamp) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (!host_buf) return set_error(TP_EINVAL, "buf is NULL");
  if (b->pf_pending) return set_error(TP_EBUSY, "beam %d already holds a prefetched block", beam);
  if (nsamp < 1 || nsamp > b->B) return set_error(TP_EINVAL, "nsamp %d not in [1, %d]", nsamp, b->B);
  const tp_plan* p = b->plan;
  if (b->pushed == 0 && nsamp <= p->max_delay)
    return set_error(TP_EINVAL, "first block (%d samples) must exceed the largest delay %lld", nsamp,
                     (long long)p->max_delay);
  DeviceGuard g(e->device);
  if (!b->pf_stream) TP_CUDA_TRY(cudaStreamCreateWithFlags(&b->pf_stream, cudaStreamNonBlocking));
  const size_t es = dtype_size(p->dtype);
  const size_t dpitch = (size_t)b->pitch * es;
  // the window the next push assembles: win[0] for the first block, else
  // the one the current block does not use, after the overlap tail
  char* dst;
  if (b->pushed == 0) {
    dst = static_cast<char*>(b->win[0]);
  } else {
    dst = static_cast<char*>(b->win[b->cur ^ 1]) + (size_t)p->max_delay * es;
    TP_CUDA_TRY(cudaStreamWaitEvent(b->pf_stream, b->ev_win_free, 0));
  }
  TP_CUDA_TRY(cudaMemcpy2DAsync(dst, dpitch, host_buf, (size_t)nsamp * es, (size_t)nsamp * es, p->nchan,
                                cudaMemcpyHostToDevice, b->pf_stream));
  TP_CUDA_TRY(cudaEventRecord(b->ev_pf, b->pf_stream));
  b->pf_pending = true;
  b->pf_nsamp = nsamp;
  return TP_OK;
}

int tp_push_prefetched(tp_engine* e, int beam) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (!b->pf_pending) return set_error(TP_ENOTREADY, "beam %d holds no prefetched block", beam);
  const int rc = check_push(b, b->pf_nsamp, beam);
  if (rc != TP_OK) return rc;
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  TP_CUDA_TRY(cudaStreamWaitEvent(s, b->ev_pf, 0));
  const int r = assemble_window(e, b, s, nullptr, 0, b->pf_nsamp, 0);
  if (r == TP_OK) b->pf_pending = false;
  return r;
}

int tp_dedisperse(tp_engine* e, int beam) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  if (beam >= 0) {
    Beam* b = get_beam(e, beam);
    if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
    return issue_dedisperse(e, b);
  }
  BatchPlan bp = plan_batch(e);
  if (bp.beams.empty()) return set_error(TP_ENOTREADY, "no beam holds a new block");
  const size_t need = batch_bytes(bp);
  if (need > kBatchBytes) return set_error(TP_EINVAL, "batch of %zu beams too large", bp.beams.size());
  int rc = wait_pushes(e, bp);
  if (rc) return rc;
  pack_batch(bp, &e->h_batch);
  TP_CUDA_TRY(cudaMemcpyAsync(e->d_batch, e->h_batch.data(), need, cudaMemcpyHostToDevice, e->stream));
  return issue_batch(e, bp, e->d_batch, false);
}

int tp_detect(tp_engine* e, int beam) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  if (beam >= 0) {
    Beam* b = get_beam(e, beam);
    if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
    return issue_detect(e, b, beam_stream(e, b));
  }
  int n = 0;
  for (Beam* b : e->beams)
    if (b && b->state == kDedispersed) {
      int rc = issue_detect(e, b, e->stream);
      if (rc) return rc;
      ++n;
    }
  return n ? TP_OK : set_error(TP_ENOTREADY, "no beam is dedispersed");
}

int tp_run_ready(tp_engine* e, int use_graph, int* nbeams) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  BatchPlan bp = plan_batch(e);
  if (nbeams) *nbeams = (int)bp.beams.size();
  if (bp.beams.empty()) return set_error(TP_ENOTREADY, "no beam holds a new block");
  const size_t need = batch_bytes(bp);
  if (need > kBatchBytes) return set_error(TP_EINVAL, "batch of %zu beams too large", bp.beams.size());
  int rc0 = wait_pushes(e, bp);
  if (rc0) return rc0;
  if (!use_graph) {
    pack_batch(bp, &e->h_batch);
    TP_CUDA_TRY(cudaMemcpyAsync(e->d_batch, e->h_batch.data(), need, cudaMemcpyHostToDevice, e->stream));
    return issue_batch(e, bp, e->d_batch, true);
  }
  if (!e->stream) return set_error(TP_EINVAL, "graphs need a non-default engine stream");
  auto it = e->graphs.find(bp.key);
  if (it == e->graphs.end()) {
    GraphEntry ge;
    TP_CUDA_TRY(cudaMalloc(&ge.d_args, need));
    pack_batch(bp, &e->h_batch);
    TP_CUDA_TRY(cudaMemcpy(ge.d_args, e->h_batch.data(), need, cudaMemcpyHostToDevice));
    // capture a copy of the states: issuing advances them
    std::vector<BeamState> st;
    for (Beam* b : bp.beams) st.push_back(b->state);
    const bool prof = e->profiling;
    e->profiling = false;
    TP_CUDA_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    const uint64_t l0 = e->launches;
    int rc = issue_batch(e, bp, ge.d_args, true);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
    e->profiling = prof;
    e->launches = l0;
    for (size_t i = 0; i < bp.beams.size(); ++i) bp.beams[i]->state = st[i];
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      cudaFree(ge.d_args);
      return rc;
    }
    if (ce != cudaSuccess) {
      cudaFree(ge.d_args);
      return cuda_error(ce, "cudaStreamEndCapture");
    }
    ce = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      cudaFree(ge.d_args);
      return cuda_error(ce, "cudaGraphInstantiate");
    }
    if (e->graphs.size() >= kMaxGraphs) {
      // a bounded cache: in-place windows make the key change with the
      // caller's buffers
      TP_CUDA_TRY(cudaStreamSynchronize(e->stream));
      for (auto& kv : e->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaFree(kv.second.d_args);
      }
      e->graphs.clear();
    }
    it = e->graphs.emplace(bp.key, ge).first;
  }
  TP_CUDA_TRY(cudaGraphLaunch(it->second.exec, e->stream));
  // the graph ran every stage of every beam of the batch
  uint64_t nl = 0;
  for (Beam* b : bp.beams) nl += 4 + 4;
  nl += bp.groups.size();
  e->launches += nl;
  for (size_t i = 0; i < bp.beams.size(); ++i) {
    Beam* b = bp.beams[i];
    b->ntt = bp.args[i].ntt;
    b->state = kDetected;
    TP_CUDA_TRY(cudaEventRecord(b->ev_detect, e->stream));
  }
  return TP_OK;
}

int tp_get_candidates(tp_engine* e, int beam, tp_candidate* out, int cap, int* n_total) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d: detection not issued", beam);
  if (cap < 0 || (cap > 0 && !out)) return set_error(TP_EINVAL, "bad output buffer");
  DeviceGuard g(e->device);
  TP_CUDA_TRY(cudaEventSynchronize(b->ev_detect));
  int status = 0;
  TP_CUDA_TRY(cudaMemcpy(&status, b->status, 4, cudaMemcpyDeviceToHost));
  if (status != 0) {
    TP_CUDA_TRY(cudaMemset(b->status, 0, 4));
    return set_error(status, status == TP_EBOUNDS ? "beam %d: a device-side bounds check failed (status %d)"
                                                  : "beam %d: a device-side wait gave up (status %d)",
                     beam, status);
  }
  unsigned long long tot = 0;
  TP_CUDA_TRY(cudaMemcpy(&tot, b->n_total, 8, cudaMemcpyDeviceToHost));
  const unsigned long long kept = std::min<unsigned long long>(tot, (unsigned long long)b->cap);
  const int ncopy = (int)std::min<unsigned long long>(kept, (unsigned long long)cap);
  if (ncopy > 0) TP_CUDA_TRY(cudaMemcpy(out, b->cand, (size_t)ncopy * sizeof(tp_candidate), cudaMemcpyDeviceToHost));
  if (n_total) *n_total = (int)std::min<unsigned long long>(tot, 0x7fffffffull);
  if (tot > (unsigned long long)b->cap)
    return set_error(TP_EOVERFLOW, "beam %d found %llu candidates, capacity %d", beam, tot, b->cap);
  if (tot > (unsigned long long)cap) return set_error(TP_ETRUNC, "%llu candidates, buffer holds %d", tot, cap);
  return TP_OK;
}

namespace {

// Memory device `dev` may write: page-locked (or registered) host memory,
// its own device memory, managed memory.
bool device_writable(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == dev;
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeManaged;
}

}  // namespace

int tp_export_candidates(tp_engine* e, int beam, tp_candidate* out, int cap, unsigned long long* n_total, int* status) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d: detection not issued", beam);
  if (cap < 0 || !n_total || (cap > 0 && !out)) return set_error(TP_EINVAL, "bad output buffers");
  if ((reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(n_total)) % 8 != 0 ||
      reinterpret_cast<uintptr_t>(status) % 4 != 0)
    return set_error(TP_EINVAL, "output buffers must be aligned (records and count to 8 bytes, status to 4)");
  DeviceGuard g(e->device);
  if ((cap > 0 && !device_writable(out, e->device)) || !device_writable(n_total, e->device) ||
      (status && !device_writable(status, e->device)))
    return set_error(TP_EINVAL, "outputs must be page-locked host memory or the engine device's memory");
  int dev_sms = 0;
  TP_CUDA_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, e->device));
  TP_CUDA_TRY(launch_export_candidates(b->cand, b->n_total, b->cap, b->status, out, cap, n_total, status, 2 * dev_sms,
                                       beam_stream(e, b)));
  e->launches += 1;
  return TP_OK;
}

namespace {

// Saved stream state of a beam (tp_beam_export / tp_beam_import): this
// header, then the overlap tail [nchan][max_delay] in the sample format, then
// (running statistics) the running means and variances, nchan doubles each.
struct BeamStateHeader {
  char magic[4];
  uint32_t version;
  int32_t nchan, ndm, dtype, max_delay;
  uint64_t delay_sum;  // sum of the plan's delay table: a plan mismatch check
  int64_t pushed, nblocks;
  double run_alpha;
  uint64_t tail_bytes, run_bytes;
};

uint64_t delay_sum(const tp_plan* p) {
  uint64_t v = 0;
  for (int32_t d : p->h_delay) v = v * 1000003u + (uint32_t)d;
  return v;
}

}  // namespace

int tp_beam_export(tp_engine* e, int beam, void* out, size_t cap, size_t* size) {
  TP_NVTX_RANGE();
  if (!e || !size) return set_error(TP_EINVAL, "engine or size is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  const tp_plan* p = b->plan;
  const size_t es = dtype_size(p->dtype);
  const size_t tail = (size_t)p->nchan * (size_t)p->max_delay * es;
  const bool run = p->run_alpha < 1.0;
  const size_t runb = run ? (size_t)p->nchan * 16 : 0;
  *size = sizeof(BeamStateHeader) + tail + runb;
  if (!out) return TP_OK;
  if (cap < *size) return set_error(TP_EINVAL, "buffer of %zu bytes, %zu needed", cap, *size);
  if (b->pushed == 0) return set_error(TP_ENOTREADY, "beam %d holds no block yet", beam);
  if (b->state != kDetected) return set_error(TP_EBUSY, "beam %d: export between blocks (after detection)", beam);
  if (b->pf_pending) return set_error(TP_EBUSY, "beam %d holds a prefetched block", beam);
  DeviceGuard g(e->device);
  TP_CUDA_TRY(cudaStreamSynchronize(beam_stream(e, b)));
  TP_CUDA_TRY(cudaStreamSynchronize(e->stream));
  BeamStateHeader h{};
  std::memcpy(h.magic, "TPBS", 4);
  h.version = 1;
  h.nchan = p->nchan;
  h.ndm = p->ndm;
  h.dtype = p->dtype;
  h.max_delay = p->max_delay;
  h.delay_sum = delay_sum(p);
  h.pushed = b->pushed;
  h.nblocks = b->nblocks;
  h.run_alpha = p->run_alpha;
  h.tail_bytes = tail;
  h.run_bytes = runb;
  unsigned char* o = static_cast<unsigned char*>(out);
  std::memcpy(o, &h, sizeof h);
  if (tail) {
    const size_t rowb = (size_t)p->max_delay * es;
    const char* src = static_cast<const char*>(b->xwin) + (size_t)(b->nsamp_win - p->max_delay) * es;
    TP_CUDA_TRY(cudaMemcpy2D(o + sizeof h, rowb, src, (size_t)b->xpitch * es, rowb, p->nchan, cudaMemcpyDeviceToHost));
  }
  if (run) {
    const int cur = (int)(b->nblocks & 1);
    TP_CUDA_TRY(cudaMemcpy(o + sizeof h + tail, b->run_mu[cur], (size_t)p->nchan * 8, cudaMemcpyDeviceToHost));
    TP_CUDA_TRY(cudaMemcpy(o + sizeof h + tail + (size_t)p->nchan * 8, b->run_var[cur], (size_t)p->nchan * 8,
                           cudaMemcpyDeviceToHost));
  }
  return TP_OK;
}

int tp_beam_import(tp_engine* e, int beam, const void* in, size_t size) {
  TP_NVTX_RANGE();
  if (!e || !in) return set_error(TP_EINVAL, "engine or state is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->pushed != 0) return set_error(TP_EBUSY, "beam %d has received blocks: import into a fresh beam", beam);
  const tp_plan* p = b->plan;
  if (size < sizeof(BeamStateHeader)) return set_error(TP_EINVAL, "state of %zu bytes is too short", size);
  BeamStateHeader h;
  std::memcpy(&h, in, sizeof h);
  if (std::memcmp(h.magic, "TPBS", 4) != 0 || h.version != 1) return set_error(TP_EINVAL, "not a beam state");
  const size_t es = dtype_size(p->dtype);
  const size_t tail = (size_t)p->nchan * (size_t)p->max_delay * es;
  const bool run = p->run_alpha < 1.0;
  const size_t runb = run ? (size_t)p->nchan * 16 : 0;
  if (h.nchan != p->nchan || h.ndm != p->ndm || h.dtype != p->dtype || h.max_delay != p->max_delay ||
      h.delay_sum != delay_sum(p))
    return set_error(TP_EINVAL, "the state was saved under a different plan");
  if (h.run_alpha != p->run_alpha) return set_error(TP_EINVAL, "the state's running-statistics weight differs");
  if (h.tail_bytes != tail || h.run_bytes != runb || size < sizeof h + tail + runb || h.pushed <= 0 ||
      h.nblocks <= 0)
    return set_error(TP_EINVAL, "inconsistent beam state");
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  const unsigned char* src = static_cast<const unsigned char*>(in);
  if (tail) {
    const size_t rowb = (size_t)p->max_delay * es;
    TP_CUDA_TRY(cudaMemcpy2DAsync(b->win[0], (size_t)b->pitch * es, src + sizeof h, rowb, rowb, p->nchan,
                                  cudaMemcpyHostToDevice, s));
  }
  if (run) {
    const int cur = (int)(h.nblocks & 1);
    TP_CUDA_TRY(cudaMemcpyAsync(b->run_mu[cur], src + sizeof h + tail, (size_t)p->nchan * 8,
                                cudaMemcpyHostToDevice, s));
    TP_CUDA_TRY(cudaMemcpyAsync(b->run_var[cur], src + sizeof h + tail + (size_t)p->nchan * 8,
                                (size_t)p->nchan * 8, cudaMemcpyHostToDevice, s));
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));  // the caller's buffer may go once we return
  // the window now holds only the overlap tail: the next push continues the
  // stream from it exactly as after the exported block
  b->cur = 0;
  b->xwin = b->win[0];
  b->xpitch = b->pitch;
  b->nsamp_win = p->max_delay;
  b->nout = 0;
  b->pushed = h.pushed;
  b->nblocks = h.nblocks;
  b->t0_abs = h.pushed - p->max_delay;
  b->state = kEmpty;
  return TP_OK;
}

int tp_beam_info(tp_engine* e, int beam, int64_t* nsamp_window, int64_t* nout, int64_t* t0_abs, int* nchunk) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  const int W = b->plan->rfi.chunk_width;
  if (nsamp_window) *nsamp_window = b->nsamp_win;
  if (nout) *nout = b->nout;
  if (t0_abs) *t0_abs = b->t0_abs;
  if (nchunk) *nchunk = (int)((b->nsamp_win + W - 1) / W);
  return TP_OK;
}

int tp_get_series(tp_engine* e, int beam, void* out, size_t bytes, int out_is_device) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state < kDedispersed) return set_error(TP_ENOTREADY, "beam %d is not dedispersed", beam);
  const size_t row = (size_t)b->nout * 4;
  if (!out || bytes < row * b->plan->ndm) return set_error(TP_EINVAL, "need %zu bytes", row * b->plan->ndm);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  TP_CUDA_TRY(cudaMemcpy2DAsync(out, row, b->D, (size_t)b->dpitch * 4, row, b->plan->ndm,
                                out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
}

int tp_get_bandpass(tp_engine* e, int beam, double* mu, double* sigma, int nchan) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (nchan != b->plan->nchan) return set_error(TP_EINVAL, "nchan %d != %d", nchan, b->plan->nchan);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  if (mu) TP_CUDA_TRY(cudaMemcpyAsync(mu, b->mu, nchan * 8, cudaMemcpyDeviceToHost, s));
  if (sigma) TP_CUDA_TRY(cudaMemcpyAsync(sigma, b->sigma, nchan * 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
}

int tp_get_masks(tp_engine* e, int beam, uint8_t* chunk_flag, uint8_t* chunk_raw, uint8_t* spec_flag) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state < kDedispersed) return set_error(TP_ENOTREADY, "beam %d is not dedispersed", beam);
  const tp_plan* p = b->plan;
  const int W = p->rfi.chunk_width;
  const size_t nk = (size_t)((b->nsamp_win + W - 1) / W);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  if (chunk_flag) TP_CUDA_TRY(cudaMemcpyAsync(chunk_flag, b->chunk_flag, p->nchan * nk, cudaMemcpyDeviceToHost, s));
  if (chunk_raw) TP_CUDA_TRY(cudaMemcpyAsync(chunk_raw, b->chunk_raw, p->nchan * nk, cudaMemcpyDeviceToHost, s));
  std::vector<uint32_t> bits;
  if (spec_flag) {
    bits.resize((size_t)((b->nsamp_win + 31) / 32));
    TP_CUDA_TRY(cudaMemcpyAsync(bits.data(), b->spec_bits, bits.size() * 4, cudaMemcpyDeviceToHost, s));
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  if (spec_flag)
    for (int64_t t = 0; t < b->nsamp_win; ++t) spec_flag[t] = (uint8_t)((bits[t >> 5] >> (t & 31)) & 1u);
  return TP_OK;
}

int tp_get_series_stats(tp_engine* e, int beam, double* mu, double* sigma, int ndm) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d: detection not issued", beam);
  if (ndm != b->plan->ndm) return set_error(TP_EINVAL, "ndm %d != %d", ndm, b->plan->ndm);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  if (mu) TP_CUDA_TRY(cudaMemcpyAsync(mu, b->row_mu, ndm * 8, cudaMemcpyDeviceToHost, s));
  if (sigma) TP_CUDA_TRY(cudaMemcpyAsync(sigma, b->row_sigma, ndm * 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
}

}  // extern "C"

extern "C" {

int tp_set_profiling(tp_engine* e, int enable) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  e->profiling = enable != 0;
  if (e->profiling) {
    DeviceGuard g(e->device);
    for (auto& ev : e->bev_pending) {
      cudaEventSynchronize(ev.second);
      e->bev_pool.push_back(ev);
    }
    e->bev_pending.clear();
    e->batch_ms = 0.0;
    e->batch_count = 0;
  }
  if (e->profiling)
    for (Beam* b : e->beams)
      if (b) {
        DeviceGuard g(e->device);
        prof_harvest(b, true);
        for (double& v : b->stage_ms) v = 0.0;
        b->stage_count = 0;
      }
  return TP_OK;
}

int tp_get_stage_times(tp_engine* e, int beam, double* ms, int64_t* count) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  DeviceGuard g(e->device);
  prof_harvest(b, true);
  if (ms)
    for (int i = 0; i < 4; ++i) ms[i] = b->stage_ms[i];
  if (count) *count = b->stage_count;
  return TP_OK;
}

int tp_engine_set_wait_limit(tp_engine* e, long long tries) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  e->wait_tries = tries < 0 ? kDefaultWaitTries : (tries > 0x7fffffffLL ? 0x7fffffffLL : tries);
  // graphs captured earlier hold the old limit in their arguments
  TP_CUDA_TRY(cudaStreamSynchronize(e->stream));
  for (auto& kv : e->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaFree(kv.second.d_args);
  }
  e->graphs.clear();
  return TP_OK;
}

int tp_engine_set_batch_grid(tp_engine* e, int ctas) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  e->batch_grid = ctas;
  TP_CUDA_TRY(cudaStreamSynchronize(e->stream));
  for (auto& kv : e->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaFree(kv.second.d_args);
  }
  e->graphs.clear();
  return TP_OK;
}

int tp_engine_set_canaries(tp_engine* e, int enable) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  e->canaries = enable != 0;
  return TP_OK;
}

int tp_engine_check_canaries(tp_engine* e, int* nbad) {
  TP_NVTX_RANGE();
  if (!e || !nbad) return set_error(TP_EINVAL, "engine or nbad is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  *nbad = 0;
  // every stream of the engine's beams may still write: wait for the device
  TP_CUDA_TRY(cudaDeviceSynchronize());
  std::vector<unsigned char> buf;
  for (Beam* b : e->beams) {
    if (!b) continue;
    for (const auto& c : b->canaries) {
      const size_t tail = round_up(std::max<size_t>(c.second, 1), 256) - c.second + kCanaryBytes;
      buf.resize(kCanaryBytes + tail);
      TP_CUDA_TRY(cudaMemcpy(buf.data(), c.first - kCanaryBytes, kCanaryBytes, cudaMemcpyDeviceToHost));
      TP_CUDA_TRY(cudaMemcpy(buf.data() + kCanaryBytes, c.first + c.second, tail, cudaMemcpyDeviceToHost));
      bool head_ok = true, tail_ok = true;
      for (size_t i = 0; i < kCanaryBytes; ++i) head_ok = head_ok && buf[i] == kCanaryByte;
      for (size_t i = 0; i < tail; ++i) tail_ok = tail_ok && buf[kCanaryBytes + i] == kCanaryByte;
      *nbad += (head_ok ? 0 : 1) + (tail_ok ? 0 : 1);
    }
  }
  return TP_OK;
}

int tp_debug_bounds(void) { return kDebugBounds ? 1 : 0; }

int tp_debug_limit_staged(tp_engine* e, int beam, int64_t bytes) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  if (!kDebugBounds) return set_error(TP_EINVAL, "not the bounds-checking build of the library");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  b->dbg_y_bytes = bytes < 0 ? -1 : bytes;
  b->h_args_valid = false;
  return TP_OK;
}

int tp_get_batch_times(tp_engine* e, double* ms, int64_t* count) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  for (auto& ev : e->bev_pending) {
    TP_CUDA_TRY(cudaEventSynchronize(ev.second));
    float t = 0.f;
    TP_CUDA_TRY(cudaEventElapsedTime(&t, ev.first, ev.second));
    e->batch_ms += t;
    e->batch_count += 1;
    e->bev_pool.push_back(ev);
  }
  e->bev_pending.clear();
  if (ms) *ms = e->batch_ms;
  if (count) *count = e->batch_count;
  return TP_OK;
}

int tp_engine_launches(const tp_engine* e, uint64_t* n) {
  if (!e || !n) return set_error(TP_EINVAL, "engine or n is NULL");
  *n = e->launches;
  return TP_OK;
}

}  // extern "C"

extern "C" {

int tp_plan_set_clustering(tp_plan* p, const tp_cluster_params* prm) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  std::lock_guard<std::recursive_mutex> lk(p->e->mu);
  if (prm) {
    if (prm->t_eps < 0 || prm->dm_eps < 0 || !(prm->snr_eps >= 0.0) || prm->min_pts < 1 || prm->smooth < 1 ||
        prm->smooth % 2 == 0 || !std::isfinite(prm->rmse_max) || !std::isfinite(prm->dm_min) ||
        !std::isfinite(prm->snr_eps))
      return set_error(TP_EINVAL, "invalid clustering parameters");
  }
  if (prm && p->ndm > tp::kMaxClusterDm)
    return set_error(TP_EINVAL, "clustering supports at most %d DM trials (plan has %d)", tp::kMaxClusterDm, p->ndm);
  if (p->users > 0) return set_error(TP_EBUSY, "plan is used by %d open beams", p->users);
  p->cluster = prm != nullptr;
  if (prm) p->cparams = *prm;
  return TP_OK;
}

int tp_get_clusters(tp_engine* e, int beam, tp_cluster* out, int cap, int* n, int* truncated) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (!b->plan->cluster) return set_error(TP_EINVAL, "the beam's plan does not cluster");
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d has no detected block", beam);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  int hn[2] = {0, 0};
  TP_CUDA_TRY(cudaMemcpyAsync(hn, b->n_clusters, 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  const int k = cap < hn[0] ? (cap > 0 ? cap : 0) : hn[0];
  if (k > 0 && out)
    TP_CUDA_TRY(cudaMemcpyAsync(out, b->clusters, (size_t)k * sizeof(tp_cluster), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  if (n) *n = hn[0];
  if (truncated) *truncated = hn[1];
  return TP_OK;
}

int tp_get_candidate_labels(tp_engine* e, int beam, int32_t* labels, int cap, int* n) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (!b->plan->cluster) return set_error(TP_EINVAL, "the beam's plan does not cluster");
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d has no detected block", beam);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  unsigned long long tot = 0;
  TP_CUDA_TRY(cudaMemcpyAsync(&tot, b->n_total, 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  const int stored = tot < (unsigned long long)b->cap ? (int)tot : b->cap;
  const int k = cap < stored ? (cap > 0 ? cap : 0) : stored;
  if (k > 0 && labels)
    TP_CUDA_TRY(cudaMemcpyAsync(labels, b->cl_label, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  if (n) *n = stored;
  return TP_OK;
}

int tp_plan_set_bandpass_fit(tp_plan* p, int order, double tau_mask) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  std::lock_guard<std::recursive_mutex> lk(p->e->mu);
  if (order < -1 || order > kMaxFitOrder) return set_error(TP_EINVAL, "fit order %d: -1 (off) .. %d", order, kMaxFitOrder);
  if (order >= 0) {
    if (!(tau_mask > 0.0) || !std::isfinite(tau_mask)) return set_error(TP_EINVAL, "tau_mask must be > 0");
    if (p->rfi.stats_mode != TP_STATS_BLOCK) return set_error(TP_EINVAL, "the fit needs block statistics");
    if (p->run_alpha < 1.0) return set_error(TP_EINVAL, "the fit and running statistics exclude each other");
    if (p->nchan > kMaxFitChannels) return set_error(TP_EINVAL, "the fit takes at most %d channels", kMaxFitChannels);
  }
  if (p->users > 0) return set_error(TP_EBUSY, "plan is used by %d open beams", p->users);
  p->fit_order = order;
  p->tau_mask = tau_mask;
  return TP_OK;
}

int tp_plan_set_running_stats(tp_plan* p, double alpha) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  std::lock_guard<std::recursive_mutex> lk(p->e->mu);
  if (!(alpha > 0.0) || !(alpha <= 1.0)) return set_error(TP_EINVAL, "alpha must lie in (0, 1]");
  if (alpha < 1.0) {
    if (p->rfi.stats_mode != TP_STATS_BLOCK) return set_error(TP_EINVAL, "running statistics need block statistics");
    if (p->fit_order >= 0) return set_error(TP_EINVAL, "the fit and running statistics exclude each other");
  }
  if (p->users > 0) return set_error(TP_EBUSY, "plan is used by %d open beams", p->users);
  p->run_alpha = alpha;
  return TP_OK;
}

int tp_get_bandpass_fit(tp_engine* e, int beam, double* bfit, uint8_t* masked, double* rmse, int nchan) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->plan->fit_order < 0) return set_error(TP_EINVAL, "the beam's plan does not fit its bandpass");
  if (b->state < kDedispersed) return set_error(TP_ENOTREADY, "beam %d has no processed block", beam);
  if (nchan != b->plan->nchan) return set_error(TP_EINVAL, "nchan %d != %d", nchan, b->plan->nchan);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  if (bfit) TP_CUDA_TRY(cudaMemcpyAsync(bfit, b->bfit, (size_t)nchan * 8, cudaMemcpyDeviceToHost, s));
  if (masked) TP_CUDA_TRY(cudaMemcpyAsync(masked, b->fit_masked, (size_t)nchan, cudaMemcpyDeviceToHost, s));
  if (rmse) TP_CUDA_TRY(cudaMemcpyAsync(rmse, b->rmse, 8, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
}

int tp_plan_set_postprocess(tp_plan* p, int median_width, int detrend) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  std::lock_guard<std::recursive_mutex> lk(p->e->mu);
  if (median_width < 1 || median_width > kMaxMedianWidth || median_width % 2 == 0)
    return set_error(TP_EINVAL, "median width %d: odd, 1..%d", median_width, kMaxMedianWidth);
  if (detrend != 0 && detrend != 1) return set_error(TP_EINVAL, "detrend must be 0 or 1");
  if (p->users > 0) return set_error(TP_EBUSY, "plan is used by %d open beams", p->users);
  p->median_width = median_width;
  p->detrend = detrend;
  return TP_OK;
}

int tp_get_processed_series(tp_engine* e, int beam, void* out, size_t bytes, int out_is_device) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d has no detected block", beam);
  const size_t row = (size_t)b->nout * 4;
  if (!out || bytes < row * (size_t)b->plan->ndm) return set_error(TP_EINVAL, "output buffer too small");
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  const void* src = b->plan->median_width > 1 ? b->M : b->D;
  TP_CUDA_TRY(cudaMemcpy2DAsync(out, row, src, (size_t)b->dpitch * 4, row, b->plan->ndm,
                                out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
}

int tp_get_detrend(tp_engine* e, int beam, double* mean, double* beta, double* sigma, int ndm) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->state != kDetected) return set_error(TP_ENOTREADY, "beam %d has no detected block", beam);
  if (!b->plan->detrend) return set_error(TP_EINVAL, "the beam's plan does not detrend");
  if (ndm < b->plan->ndm) return set_error(TP_EINVAL, "ndm %d < %d", ndm, b->plan->ndm);
  DeviceGuard g(e->device);
  cudaStream_t s = beam_stream(e, b);
  const size_t nb = (size_t)b->plan->ndm * 8;
  if (mean) TP_CUDA_TRY(cudaMemcpyAsync(mean, b->row_mu, nb, cudaMemcpyDeviceToHost, s));
  if (beta) TP_CUDA_TRY(cudaMemcpyAsync(beta, b->row_beta, nb, cudaMemcpyDeviceToHost, s));
  if (sigma) TP_CUDA_TRY(cudaMemcpyAsync(sigma, b->row_sigma, nb, cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
}

int tp_plan_shapes(const tp_plan* p, int* shape, int* feasible, int n) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  if (shape) *shape = p->shape;
  if (feasible)
    for (int i = 0; i < n && i < kNumShapes; ++i) feasible[i] = p->feasible[i] ? 1 : 0;
  return kNumShapes;
}

int tp_plan_set_shape(tp_plan* p, int shape) {
  if (!p) return set_error(TP_EINVAL, "plan is NULL");
  if (shape < 0 || shape >= kNumShapes || !p->feasible[shape])
    return set_error(TP_EINVAL, "shape %d is not feasible for this plan", shape);
  std::lock_guard<std::recursive_mutex> lk(p->e->mu);
  p->shape = shape;
  p->h_tiles = p->shape_tiles[shape];
  p->d_tiles = p->d_shape_tiles[shape];
  return TP_OK;
}

int tp_autotune_batch(tp_engine* e, int reps, int* best, float* ms, int n) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  DeviceGuard g(e->device);
  std::vector<Beam*> bs;
  for (Beam* b : e->beams)
    if (b && b->nsamp_win > 0) bs.push_back(b);
  if (bs.empty()) return set_error(TP_ENOTREADY, "no beam has received a block");
  const size_t need = bs.size() * sizeof(DedispArgs) + 2 * sizeof(int) + bs.size() * sizeof(int) + 16;
  if (need > kBatchBytes) return set_error(TP_EINVAL, "batch of %zu beams too large", bs.size());
  // the beams grouped by plan: each plan gets its own kernel shape
  std::vector<tp_plan*> plans;
  std::vector<std::vector<Beam*>> groups;
  std::vector<double> work;
  for (Beam* b : bs) {
    tp_plan* p = const_cast<tp_plan*>(b->plan);
    size_t k = 0;
    while (k < plans.size() && plans[k] != p) ++k;
    if (k == plans.size()) {
      plans.push_back(p);
      groups.emplace_back();
      work.push_back(0.0);
    }
    groups[k].push_back(b);
    work[k] += (double)p->ndm * (double)p->nchan * (double)b->nout;
  }
  // every earlier block of every beam is finished before the timing runs
  for (Beam* b : bs) TP_CUDA_TRY(cudaStreamSynchronize(beam_stream(e, b)));
  TP_CUDA_TRY(cudaStreamSynchronize(e->stream));
  cudaStream_t s = e->stream;
  cudaEvent_t e0, e1;
  TP_CUDA_TRY(cudaEventCreate(&e0));
  TP_CUDA_TRY(cudaEventCreate(&e1));
  reps = reps < 1 ? 1 : reps;
  std::vector<unsigned char> buf;
  // ms of the batched launch of group k with shape sh (-1: not feasible)
  std::vector<std::vector<float>> t(plans.size(), std::vector<float>(kNumShapes, -1.f));
  for (int sh = 0; sh < kNumShapes; ++sh)
    for (size_t k = 0; k < plans.size(); ++k) {
      if (!plans[k]->feasible[sh]) continue;
      std::vector<DedispArgs> args;
      std::vector<int> cta{0};
      bool ok = true;
      for (Beam* b : groups[k]) {
        DedispArgs da = dedisp_args(b->plan, b);
        da.shape = sh;
        da.tiles = b->plan->d_shape_tiles[sh];
        da.ntiles = (int)b->plan->shape_tiles[sh].size();
        da.ntt = (int)((b->nout + shape_tile_t(sh) - 1) / shape_tile_t(sh));
        if (da.ntt > b->ntt_max) ok = false;
        args.push_back(da);
        cta.push_back(cta.back() + da.ntiles * da.ntt);
      }
      if (!ok) continue;
      buf.resize(args.size() * sizeof(DedispArgs) + cta.size() * sizeof(int));
      std::memcpy(buf.data(), args.data(), args.size() * sizeof(DedispArgs));
      std::memcpy(buf.data() + args.size() * sizeof(DedispArgs), cta.data(), cta.size() * sizeof(int));
      TP_CUDA_TRY(cudaMemcpyAsync(e->d_batch, buf.data(), buf.size(), cudaMemcpyHostToDevice, s));
      BatchArgs ba{static_cast<const DedispArgs*>(e->d_batch),
                   reinterpret_cast<const int*>(static_cast<unsigned char*>(e->d_batch) +
                                                args.size() * sizeof(DedispArgs)),
                   (int)args.size(), e->d_items, e->wait_tries};
      const int dtype = plans[k]->dtype;
      TP_CUDA_TRY(cudaMemsetAsync(e->d_items, 0, sizeof(int), s));
      TP_CUDA_TRY(launch_dedisperse(sh, dtype, ba, cta.back(), s, e->batch_grid));  // warm-up
      TP_CUDA_TRY(cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r) {
        TP_CUDA_TRY(cudaMemsetAsync(e->d_items, 0, sizeof(int), s));
        TP_CUDA_TRY(launch_dedisperse(sh, dtype, ba, cta.back(), s, e->batch_grid));
      }
      TP_CUDA_TRY(cudaEventRecord(e1, s));
      TP_CUDA_TRY(cudaEventSynchronize(e1));
      e->launches += 1 + reps;
      float tt = 0.f;
      TP_CUDA_TRY(cudaEventElapsedTime(&tt, e0, e1));
      t[k][sh] = tt / reps;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // each plan's fastest shape; the whole batch's time per shape where every
  // plan admits it
  int bestsh = -1;
  size_t heaviest = 0;
  for (size_t k = 0; k < plans.size(); ++k) {
    int pk = -1;
    for (int sh = 0; sh < kNumShapes; ++sh)
      if (t[k][sh] >= 0.f && (pk < 0 || t[k][sh] < t[k][pk])) pk = sh;
    if (pk < 0) return set_error(TP_EINVAL, "no kernel shape is feasible for a plan of the batch");
    tp_plan_set_shape(plans[k], pk);
    if (work[k] > work[heaviest]) heaviest = k;
    if (k == heaviest) bestsh = pk;
  }
  for (size_t k = 0; k < plans.size(); ++k)
    if (k == heaviest) bestsh = plans[k]->shape;
  if (ms)
    for (int sh = 0; sh < kNumShapes && sh < n; ++sh) {
      float sum = 0.f;
      bool all = true;
      for (size_t k = 0; k < plans.size(); ++k) {
        if (t[k][sh] < 0.f) all = false;
        sum += t[k][sh];
      }
      ms[sh] = all ? sum : -1.f;
    }
  // the timing runs overwrote the series: each beam must be dedispersed again
  for (Beam* b : bs)
    if (b->state >= kDedispersed) b->state = kReady;
  if (best) *best = bestsh;
  return TP_OK;
}

}  // extern "C"

namespace {

// The autotuner cache file: one entry per line, "key" shape ms.  Keys hold
// no quote and no newline.
void tune_load(tp_engine* e) {
  e->tune_cache.clear();
  FILE* f = std::fopen(e->tune_path.c_str(), "r");
  if (!f) return;
  char line[2048];
  while (std::fgets(line, sizeof line, f)) {
    const char* q0 = std::strchr(line, '"');
    const char* q1 = q0 ? std::strchr(q0 + 1, '"') : nullptr;
    int shape = -1;
    float t = -1.f;
    if (!q1 || std::sscanf(q1 + 1, "%d %f", &shape, &t) != 2) continue;
    if (shape >= 0 && shape < kNumShapes) e->tune_cache[std::string(q0 + 1, q1)] = {shape, t};
  }
  std::fclose(f);
}

void tune_save(const tp_engine* e) {
  const std::string tmp = e->tune_path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "# dedispersion kernel shapes chosen by tp_autotune: \"key\" shape ms\n");
  for (const auto& kv : e->tune_cache) std::fprintf(f, "\"%s\" %d %.6g\n", kv.first.c_str(), kv.second.first, kv.second.second);
  std::fclose(f);
  std::rename(tmp.c_str(), e->tune_path.c_str());
}

// What the timing depends on: the device, the plan's geometry and format,
// the block's output length and the set of kernel shapes.
std::string tune_key(const tp_engine* e, const tp_plan* p, const Beam* b) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, e->device);
  uint64_t h = 1469598103934665603ull;
  for (double d : p->dm) {
    uint64_t u;
    std::memcpy(&u, &d, 8);
    h = (h ^ u) * 1099511628211ull;
  }
  char buf[512];
  std::snprintf(buf, sizeof buf, "%s cc%d.%d sms%d | nchan %d f_lo %.17g bw %.17g t_samp %.17g dtype %d ndm %d dm %016llx | "
                "nout %lld | shapes %d",
                prop.name, prop.major, prop.minor, prop.multiProcessorCount, p->nchan, p->f_lo, p->bw, p->t_samp,
                p->dtype, p->ndm, (unsigned long long)h, (long long)b->nout, kNumShapes);
  std::string k(buf);
  for (char& ch : k)
    if (ch == '"' || ch == '\n') ch = ' ';
  return k;
}

}  // namespace

extern "C" {

int tp_engine_set_tuning_cache(tp_engine* e, const char* path) {
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  e->tune_path = path ? path : "";
  e->tune_cache.clear();
  if (!e->tune_path.empty()) tune_load(e);
  return TP_OK;
}

int tp_autotune(tp_engine* e, int beam, int reps, int* best, float* ms, int n) {
  TP_NVTX_RANGE();
  if (!e) return set_error(TP_EINVAL, "engine is NULL");
  std::lock_guard<std::recursive_mutex> lk(e->mu);
  Beam* b = get_beam(e, beam);
  if (!b) return set_error(TP_EINVAL, "no beam %d", beam);
  if (b->nsamp_win == 0) return set_error(TP_ENOTREADY, "beam %d has no block yet", beam);
  tp_plan* p = const_cast<tp_plan*>(b->plan);
  DeviceGuard g(e->device);
  std::string key;
  if (!e->tune_path.empty()) {
    key = tune_key(e, p, b);
    auto it = e->tune_cache.find(key);
    if (it != e->tune_cache.end() && p->feasible[it->second.first]) {
      // a cached choice: no timing runs; as after them, the beam is to be
      // dedispersed again with the chosen shape
      if (ms)
        for (int sh = 0; sh < n; ++sh) ms[sh] = sh == it->second.first ? it->second.second : -1.f;
      if (b->state >= kDedispersed) b->state = kReady;
      tp_plan_set_shape(p, it->second.first);
      if (best) *best = it->second.first;
      return TP_OK;
    }
  }
  cudaStream_t s = beam_stream(e, b);
  cudaEvent_t e0, e1;
  TP_CUDA_TRY(cudaEventCreate(&e0));
  TP_CUDA_TRY(cudaEventCreate(&e1));
  reps = reps < 1 ? 1 : reps;
  int bestsh = -1;
  float bestms = 0.f;
  for (int sh = 0; sh < kNumShapes; ++sh) {
    if (ms && sh < n) ms[sh] = -1.f;
    if (!p->feasible[sh]) continue;
    DedispArgs da = dedisp_args(p, b);
    da.shape = sh;
    da.tiles = p->d_shape_tiles[sh];
    da.ntiles = (int)p->shape_tiles[sh].size();
    da.ntt = (int)((b->nout + shape_tile_t(sh) - 1) / shape_tile_t(sh));
    int rc = launch_single(e, b, da, sh, s);  // warm-up
    if (rc) return rc;
    TP_CUDA_TRY(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) {
      rc = launch_single(e, b, da, sh, s);
      if (rc) return rc;
    }
    TP_CUDA_TRY(cudaEventRecord(e1, s));
    TP_CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0.f;
    TP_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
    t /= reps;
    if (ms && sh < n) ms[sh] = t;
    if (bestsh < 0 || t < bestms) bestsh = sh, bestms = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timing runs overwrote the series: the beam must be dedispersed again
  if (b->state >= kDedispersed) b->state = kReady;
  tp_plan_set_shape(p, bestsh);
  if (best) *best = bestsh;
  if (!key.empty() && bestsh >= 0) {
    e->tune_cache[key] = {bestsh, bestms};
    tune_save(e);
  }
  return TP_OK;
}

}  // extern "C"
