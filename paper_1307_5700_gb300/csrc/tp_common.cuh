// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>

#include "tp_dedisp.h"

namespace tp {

// An NVTX range around one public call, named after the call (Nsight Systems
// shows it on the host timeline; `ncu --nvtx --nvtx-include "tp_detect/"`
// captures only the kernels that call launches).  With no tool attached it
// costs a function-pointer test.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define TP_NVTX_RANGE() ::tp::NvtxRange tp_nvtx_range_(__func__)

// Sets the thread's last-error text (printf-style) and returns `code`.
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t err, const char* what);

#define TP_CUDA_TRY(expr)                                         \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ::tp::cuda_error(_e, #expr);    \
  } while (0)

// ---- debug bounds checks ----------------------------------------------------------

// The debug build of the library (TP_DEBUG_BOUNDS defined, libtpdd_debug.so)
// checks the global and shared accesses of its kernels whose indices come from
// the plan's geometry, the delays or the data.  A failed check records
// TP_EBOUNDS in the beam's status word (the first error is kept) and the
// access is skipped: nothing traps, so the context stays usable and the host
// reads the code with the block's results.  The release build compiles every
// check to `true`.
#ifdef TP_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif

// [off, off + n) inside [0, extent)?  An empty range always is.  (Debug
// build; release: true.)
__device__ __forceinline__ bool in_bounds(int64_t off, int64_t n, int64_t extent, int* status) {
  if constexpr (kDebugBounds) {
    if (n == 0 || (off >= 0 && n > 0 && off + n <= extent)) return true;
    if (status) atomicCAS(status, 0, TP_EBOUNDS);
    return false;
  } else {
    return true;
  }
}

// ---- per-block device arguments ------------------------------------------------

// What the RFI kernels need about one beam's current block.
struct RfiArgs {
  const void* x;          // window, channel-major, row pitch `pitch` elements
  int64_t pitch;          // elements per channel row
  int nchan;
  int64_t nsamp;          // window length N_s
  int W;                  // chunk width W_c
  int nchunk;             // ceil(N_s / W)
  int dtype;              // TP_U8 / TP_F16 / TP_BF16 / TP_F32
  int stats_mode;         // TP_STATS_BLOCK / TP_STATS_EXTERNAL
  int enable_channel, enable_spectrum, dilate_channels;
  double tau_c, tau_s;
  // per-channel statistics (outputs in block mode, inputs in external mode)
  double* mu;             // [nchan]
  double* sigma;          // [nchan]
  long long* S;           // [nchan] exact sum (8-bit, block mode)
  long long* V;           // [nchan] N*Q - S^2 (8-bit, block mode)
  int* bint;              // [nchan] integer bandpass value (8-bit)
  float* mu_hi;           // [nchan] mu split into two floats (float data)
  float* mu_lo;
  unsigned short* b16;    // [nchan] bandpass value in the 16-bit storage format
  double* bsum;           // [1] sum over channels of the bandpass values
  // masks
  uint8_t* chunk_raw;     // [nchan][nchunk] exceedances
  uint8_t* chunk_flag;    // [nchan][nchunk] after dilation
  int* chan_nflag;        // [nchan] flagged chunks per channel
  uint32_t* spec_bits;    // [ceil(N_s/32)] spectrum flags
  int* spec_nflag;        // [1] flagged spectra
  double* spec_thr;       // [nchunk] spectrum threshold of each chunk (its unflagged channels)
  int stage_f32;          // 16-bit data: stage y = x~ - b in FP32 (for the FP32 kernel shapes)
  // fitted bandpass (Sec. 2.2.1 "Bandpass Correction"): fit = 1 turns it on
  // (0, the zero-initialised value, leaves the block statistics); the chunk
  // test then uses the fit b_c of order fit_order and its RMSE
  int fit;
  int fit_order;
  double tau_mask;        // high-power channel masking before the fit
  float* pivot;           // [nchan] per-channel pivot of the float chunk sums
  double* bfit;           // [nchan] fitted bandpass b_c
  uint8_t* fit_masked;    // [nchan] channels masked before the fit
  double* fit_work;       // [2 nchan] local excess e_c, interpolated bandpass
  double* rmse;           // [1] RMSE of the fit
  // running statistics across blocks (reading R15): run = 1 turns them on;
  // the block's statistics are folded into the previous state (run_prev_*,
  // ignored for the stream's first block) with weight run_alpha, the new
  // state goes to run_mu / run_var, and the block is then thresholded and
  // corrected with the running values
  int run;
  int run_first;
  double run_alpha;
  const double* run_prev_mu;  // [nchan]
  const double* run_prev_var; // [nchan]
  double* run_mu;             // [nchan]
  double* run_var;            // [nchan]
  // extents for the debug build's bounds checks
  int* status;                // beam status word (TP_EBOUNDS), or NULL
  int64_t x_elems;            // elements of the window buffer x
  int64_t y_elems;            // elements of the staged series
};

// Largest polynomial order and channel count of the fitted bandpass.
constexpr int kMaxFitOrder = 8;
constexpr int kMaxFitChannels = 8192;

// A tile of consecutive DM trials processed by one dedispersion CTA.
struct DmTile {
  int d0;     // first DM index
  int nd;     // number of DMs (<= kMaxTileDm)
};

struct DedispArgs {
  const void* y;          // staged series [nchan][ypitch]: FP32 y, or x~ in its storage format
  int64_t ypitch;         // samples per row (>= window + tile + 16)
  const double* bsum;     // 16-bit modes: sum over channels of the bandpass values
  int nchan;
  int64_t nout;           // T
  int dtype;
  const int32_t* delay;   // [ndm][nchan]
  const int32_t* delayT;  // [nchan][dtpitch] (transposed copy)
  int64_t dtpitch;
  int ndm;
  const DmTile* tiles;    // [ntiles]
  int ntiles;
  int ntt;                // number of time tiles
  int shape;              // index into kShapes
  void* D;                // [ndm][dpitch] float or int32
  int64_t dpitch;
  void* row_part;         // [ndm][ntt] (float: double2 {sum, sumsq}; int: longlong2)
  int* status;            // device status word (TP_ETIMEOUT on a wait that gave up)
  // extents for the debug build's bounds checks
  int64_t y_bytes;        // bytes of the staged series
  int64_t d_elems;        // elements of D
  int64_t delayT_elems;   // elements of delayT
};

// Default number of attempts of the dedispersion kernel's waits for staged
// data or a free stage buffer (each attempt is one mbarrier try_wait); the
// wait for the CTA's own copies in flight before it leaves always uses this.
constexpr long long kDefaultWaitTries = 1LL << 24;

// One launch of the dedispersion kernel covers several beams (same kernel
// shape and sample format): CTA i works for the beam b with
// cta_start[b] <= i < cta_start[b + 1], on its (i - cta_start[b])-th
// (DM tile, time tile) pair.
struct BatchArgs {
  const DedispArgs* beams;  // device, nbeams entries
  const int* cta_start;     // device, nbeams + 1 entries
  int nbeams;
  int* next_item;           // device counter, 0 at launch: CTAs past their first item take
                            // gridDim.x + atomicAdd(next_item, 1); NULL: item + gridDim.x
  long long wait_tries;     // attempts of a wait for staged data or a free stage buffer (a kernel
                            // parameter: read from the constant bank, no load in the wait path)
};

// Register-tile shapes of the dedispersion kernel.
struct KernelShape {
  int K;      // DM trials per warp
  int S;      // consecutive outputs per lane and segment (tile = 32 S samples; ALGO 4: 64 S,
              // two segments)
  int OMAX;   // largest in-window offset the kernel handles
  int NCONS;  // consumer warps per CTA (DM groups per tile)
  int FMT;    // staged series: 4 = FP32 y (FP32 data, or 16-bit float data staged as
              // FP32 x~ - b), 2 = 16-bit float x~, 3 = 8-bit x~ as 16-bit integers
  int ALGO;   // 0: register window + shifted-add dispatch; 1: direct shared loads;
              // 2: DM pairs sharing one window; 3: DM quads sharing one window;
              // 4: DM quads over two output segments with paired FP32 adds;
              // 5: DM quads with a lane's outputs s and s + S / 2 paired;
              // 6, 7, 8: 4, 5, 3 without a producer warp (consumers issue the copies)
};
constexpr int kNumShapes = 68;
extern const KernelShape kShapes[kNumShapes];
int shape_tile_t(int shape);

struct DetectArgs {
  const void* D;
  int64_t dpitch;
  int ndm;
  int64_t nout;
  int is_int;
  const void* row_part;   // as in DedispArgs
  int ntt;
  double nsigma;
  int beam;
  const long long* t0_abs;  // [1] stream index of window sample 0 (device)
  double* row_mu;         // [ndm]
  double* row_sigma;      // [ndm]
  float* row_thr_f;       // [ndm] smallest float D that is a detection
  int* row_thr_i;         // [ndm] smallest int D that is a detection
  uint32_t* hit_bits;     // [ndm][ceil(nout/32)]
  int64_t hit_pitch;      // words per row
  uint32_t* blk_count;    // [nblk]
  uint32_t* blk_off;      // [nblk]
  int nblk_t;             // CTAs per row
  tp_candidate* cand;
  int cap;
  unsigned long long* n_total;  // [1]
  // post-processing (Sec. 2.2.3): median width (1 = off), detrending; when
  // either is on, post_kernel reads D, writes the median-filtered series to M
  // (median_width > 1) and the per-(DM, 4096-sample tile) sums to post_part,
  // and the detection runs on M (or D)
  int median_width;
  int detrend;
  void* M;                // [ndm][dpitch] like D
  void* post_part;        // [ndm][nblk_t] x 3: float data double {Sy, Sdy, Syy}, int data long long
  double* row_beta;       // [ndm] detrending slope per unit of u = 2t - (T - 1)
  // extents for the debug build's bounds checks
  int* status;            // beam status word (TP_EBOUNDS)
  int64_t d_elems;        // elements of D (and of M)
  int64_t hit_elems;      // words of hit_bits
};

// Clustering of a block's detections (cluster.cu).
struct ClusterArgs {
  const tp_candidate* cand;           // (d, t)-ordered records
  const unsigned long long* n_total;  // [1] detections found
  int cap;                            // records stored
  int ndm;
  const double* dm;                   // [ndm] DM values
  double t_samp, bw_mhz, f_ghz;
  int64_t t_eps;
  int dm_eps;
  float snr_eps;
  int min_pts, smooth;
  double rmse_max, dm_min;
  int* row_start;                     // [ndm + 1]
  int* core;                          // [cap]
  int* parent;                        // [cap]
  int* root;                          // [cap]
  int* rank;                          // [cap]
  int* label;                         // [cap]
  int* order;                         // [cap] records grouped by cluster
  int max_clusters;
  int* cl_count;                      // [max_clusters]
  int* cl_offset;                     // [max_clusters + 1]
  int* cl_cursor;                     // [max_clusters]
  tp_cluster* clusters;               // [max_clusters]
  int* n_clusters;                    // [1]
  int* truncated;                     // [1]
};
cudaError_t launch_cluster(const ClusterArgs& a, cudaStream_t s);
constexpr int kMaxClusters = 65536;  // clusters kept per block
constexpr int kMaxClusterDm = 14336;  // DM trials a clustering plan may have (shared memory)

// Largest median-filter width of the post-processing.
constexpr int kMaxMedianWidth = 9;

// Dedispersion tiling constants (shared by the planner and the kernel).
constexpr int kMinTileT = 256;      // smallest output tile any shape may use (sizes buffers)
constexpr int kMaxTileT = 1472;     // largest output tile of any shape
constexpr int kMaxOverhang = 512;   // max delay spread inside a CTA tile
constexpr int kDetectT = 4096;      // samples per detection CTA

// ---- launchers (each returns a cudaError_t of the launch) -----------------------
cudaError_t launch_delay_table(int nchan, double f_lo, double bw, double t_samp, const double* dm,
                               int ndm, int32_t* delay, int* err_flag, cudaStream_t s);
cudaError_t launch_rfi(const RfiArgs& a, void* chunk_sums, void* y, int64_t ypitch,
                       cudaStream_t s, int* kernels = nullptr);
cudaError_t launch_channel_stats(const RfiArgs& a, void* chunk_sums, cudaStream_t s);
// ctas = work items; grid_limit < 0: one CTA per item, 0: a persistent grid
// (as many CTAs as are resident at once), > 0: at most that many CTAs
cudaError_t launch_dedisperse(int shape, int dtype, const BatchArgs& ba, int ctas, cudaStream_t s,
                              int grid_limit = -1);
cudaError_t launch_detect(const DetectArgs& a, cudaStream_t s);
cudaError_t launch_export_candidates(const tp_candidate* cand, const unsigned long long* n_total, int beam_cap,
                                     int* status, tp_candidate* out, int cap, unsigned long long* out_count,
                                     int* out_status, int grid, cudaStream_t s);
// Device-to-device copy of nrows rows of row_bytes bytes (pitched); a
// 16-byte vector kernel when every address, pitch and the row length are
// multiples of 16 bytes, else cudaMemcpy2DAsync.
// *kernels (may be NULL) is incremented when the kernel ran.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row_bytes, int nrows,
                      cudaStream_t s, int* kernels);

size_t dtype_size(int dtype);

}  // namespace tp
