// Entry point that allocates nothing: bandpass statistics and channel flags
// (A1-A2) with the scratch held in a fixed device array of this library.
//
// Who needs it: callers that may not allocate device memory while they run --
// for example a host process whose device memory is carved up in advance by
// a real-time scheduler, code running inside a stream capture that must not
// record allocation nodes, or an embedding runtime that forbids the CUDA
// allocator after start-up.  They pass their inputs and outputs; everything
// else lives in g_noalloc_scratch.
#include <mutex>

#include "tp_common.cuh"

namespace tp {
namespace {

// 32 MiB, kept by every device that loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is not a device address).
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(TP_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TP_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" int tp_channel_stats_noalloc(const void* x, int dtype, int nchan, int64_t nsamp, int64_t pitch,
                                        const tp_rfi_params* rfi, double* mu, double* sigma,
                                        uint8_t* chunk_flag, uint8_t* chunk_raw, void* cuda_stream) {
  if (!x || !mu || !sigma || !chunk_flag || !chunk_raw) return set_error(TP_EINVAL, "a pointer is NULL");
  if (dtype_size(dtype) == 0) return set_error(TP_EINVAL, "unknown dtype %d", dtype);
  if (nchan <= 0 || nchan > 65535 || nsamp <= 0 || pitch < nsamp) return set_error(TP_EINVAL, "bad sizes");
  tp_rfi_params r;
  if (rfi) r = *rfi;
  else tp_rfi_defaults(&r);
  if (r.chunk_width < 1) return set_error(TP_EINVAL, "chunk_width must be >= 1");
  if (r.stats_mode != TP_STATS_BLOCK)
    return set_error(TP_EINVAL, "only block statistics (the statistics are outputs here)");
  const size_t es = dtype_size(dtype);
  if (((uintptr_t)x & 15) != 0 || ((size_t)pitch * es) % 16 != 0)
    return set_error(TP_EINVAL, "x must be 16-byte aligned with a row pitch of a multiple of 16 bytes");
  const int64_t nchunk = (nsamp + r.chunk_width - 1) / r.chunk_width;
  const size_t nc = (size_t)nchan;
  // chunk sums; S, V; bint, mu_hi, mu_lo, chan_nflag; b16 (the bandpass value
  // in the 16-bit storage format, written by the binary16/bfloat16 statistics)
  const size_t need = align256(nc * (size_t)nchunk * 16) + 2 * align256(nc * 8) + 4 * align256(nc * 4) +
                      align256(nc * 2);
  if (need > kNoAllocScratchBytes)
    return set_error(TP_EINVAL, "nchan x ceil(nsamp / W) too large: needs %zu bytes of scratch, the library "
                     "holds %zu", need, kNoAllocScratchBytes);
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  auto take = [&](size_t bytes) {
    void* q = p;
    p += align256(bytes);
    return q;
  };
  RfiArgs a{};
  a.x = x;
  a.pitch = pitch;
  a.nchan = nchan;
  a.nsamp = nsamp;
  a.W = r.chunk_width;
  a.nchunk = (int)nchunk;
  a.dtype = dtype;
  a.stats_mode = TP_STATS_BLOCK;
  a.enable_channel = r.enable_channel;
  a.enable_spectrum = 0;
  a.dilate_channels = r.dilate_channels;
  a.tau_c = r.tau_channel;
  a.tau_s = r.tau_spectrum;
  void* chunk_sums = take(nc * (size_t)nchunk * 16);
  a.mu = mu;
  a.sigma = sigma;
  a.S = static_cast<long long*>(take(nc * 8));
  a.V = static_cast<long long*>(take(nc * 8));
  a.bint = static_cast<int*>(take(nc * 4));
  a.mu_hi = static_cast<float*>(take(nc * 4));
  a.mu_lo = static_cast<float*>(take(nc * 4));
  a.chan_nflag = static_cast<int*>(take(nc * 4));
  a.b16 = static_cast<unsigned short*>(take(nc * 2));
  a.chunk_raw = chunk_raw;
  a.chunk_flag = chunk_flag;
  cudaError_t e = launch_channel_stats(a, chunk_sums, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_error(e, "channel statistics kernels");
  return TP_OK;
}
