// A5: brute-force incoherent dedispersion (Sec. 2.2.2, delays of Eq. 1)
//
//   D[d][t] = sum_{c=0}^{nchan-1} y[c][t + delay[d][c]],   0 <= t < T,
//
// over the series staged by the A3/A4 kernel: FP32 y for FP32 data, else the
// stored samples x~ in their own format (binary16, bfloat16, 8-bit), whose
// sum of bandpass values the epilogue subtracts.
//
// Work decomposition.  A CTA owns a tile of consecutive DM trials (up to
// NCONS groups of K) x TT = 32 S output samples.  Consumer warp w owns group
// w; lane l owns the S consecutive outputs t0 + l S .. + S - 1 of each of the
// K DMs.  The last warp is the producer: for each pipeline stage (kNC
// channels) it stages the stage's delays for the tile's DMs and copies, per
// channel, the samples the tile needs,
// [t0 + delay[d_first][c], t0 + TT + delay[d_last][c]) rounded out to 16 B,
// with cp.async.bulk onto a "full" mbarrier; consumers release a stage on an
// "empty" mbarrier (STAGES stages in flight, no CTA-wide barrier).
//
// Consumers (ALGO 1) read each DM's S samples straight from shared memory at
// that DM's offset: FP32, one 32-bit load per add; 16-bit, S/2 + 1 words, a
// half-word shift for odd offsets, mixed-precision FP32 adds; 8-bit, S/4 + 1
// words, a byte funnel shift and two byte permutes per word that spread four
// samples into two words of 16-bit lanes, summed as packed integers (two
// channels per add) and folded into 32-bit sums every 256 channels.  ALGO 0
// instead loads one register window per channel and adds it at each DM's
// in-window offset through an indexed branch (brx.idx) into unrolled add
// sequences (dispatch_gen.cuh), reusing each loaded sample for K trials.
// ALGO 2 and 3 share one window between two or four consecutive trials
// (one indexed branch per channel selects the block for their delay steps).
// ALGO 4 is ALGO 3 with two output segments per lane, t0 + l S and
// t0 + 32 S + l S (TT = 64 S): the same window sample of both segments sits
// in one register pair and one add.rn.f32x2 updates both accumulators, which
// halves the add instructions per output; every lane still rounds each add
// to binary32 as the scalar form does.  ALGO 5 pairs a lane's own outputs
// s and s + S / 2 instead (S odd, output 2 (S / 2) added alone): register
// pair k holds window samples k and k + S / 2 of the one window, so each
// sample is loaded once for both halves.  ALGO 6 and 7 are ALGO 4 and 5
// without the producer warp: its register share goes to an eighth consumer
// warp, and consumer warp w also issues the delays and bulk copies of stages
// w, w + NCONS, ... kLookRot stages ahead of their use, over kStagesRot
// buffers, so that the warp that fills a buffer rarely waits for the others to
// release it.
// ALGO 9, 10 and 11 are ALGO 8 (8-bit quads, no producer warp) with the
// channel loop of a stage inside one assembly block: each channel's pass
// fetches the next channel's window offset and block index first, then
// issues its window loads and packed adds (9: loads before adds, the adds
// alternating between a 32-bit and a two-lane 16-bit add so that they spread
// over two execution pipes; 10: loads and adds interleaved, alternating; 11:
// interleaved, 32-bit adds only), and branches back to one indexed dispatch.
// Each (d, t) adds its channels in index order (FP32, or exact integers).
// Every mbarrier wait is bounded; a wait for staged data or a free stage
// buffer gives up after BatchArgs::wait_tries attempts, records TP_ETIMEOUT
// in the beam's status word, and the CTA leaves after letting its own copies
// land (that drain always allows kDefaultWaitTries attempts).
//
// The epilogue writes D (FP32, or int32 for 8-bit data, exact) and per
// (DM, time tile) sums of D and D^2 for the series statistics of A6.
#pragma once

#include <cstdint>
#include <type_traits>

#include "dedisp_shapes.cuh"
#include "dispatch_gen.cuh"
#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kNC = 4;                              // channels per pipeline stage
constexpr int kStages = 4;                          // pipeline depth (8-bit data: kStagesU8)
constexpr int kStagesU8 = 8;
constexpr int kStagesRot = 6;                       // ALGO 6, 7: pipeline depth
constexpr int kLookRot = 2;                         // ALGO 6, 7: stages issued ahead of use
constexpr int kDelRing = 8;                         // stages of delays prefetched ahead
constexpr long long kSpinLimit = kDefaultWaitTries;  // drain of the CTA's own copies in flight

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

// At most `tries` (< 2^31) attempts; the first, which usually succeeds, ahead
// of the loop.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long tries = kSpinLimit) {
  const int n = (int)tries;
  if (n <= 0) return false;
  if (mbar_try_wait(bar, parity)) return true;
  for (int spin = 1; spin < n; ++spin)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 4-byte asynchronous global -> shared copy; zero-fills when !valid (the
// source is not read then)
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
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
constexpr int kModeF16 = 1;   // binary16 x~
constexpr int kModeBF16 = 2;  // bfloat16 x~
constexpr int kModeU8 = 3;    // 8-bit x~ widened to 16 bits, summed as packed 16-bit integers

// 8-bit mode: channels summed into packed 16-bit lanes before they are folded
// into the 32-bit sums (256 x 255 < 2^16, so no lane can carry into the next)
constexpr int kU8FoldStages = 256 / kNC;

template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB = 1>
struct Shape {
  // ALGO 6, 7 and 8: the consumer schemes of ALGO 4, 5 and 3 without a
  // producer warp (every consumer warp issues the copies of every NCONS-th
  // stage)
  static constexpr bool ROT = ALGO >= 6;
  static constexpr int AB = ALGO >= 8 ? 3 : ROT ? ALGO - 2 : ALGO;
  // ALGO 9-11: the 8-bit quads of ALGO 8 with every channel of a stage added
  // in one call (variant ALGO - 6 of add_quad8t)
  static constexpr bool THREADED = ALGO >= 9 && ALGO <= 11;
  // ALGO 12: ALGO 8 with the copies issued four stages ahead of their use
  // over eight stage buffers (the 8-bit rows are half as long as FP32 ones)
  static constexpr int LOOK = ALGO == 12 ? 4 : kLookRot;
  static constexpr int EB = MODE == kModeF32 ? 4 : 2;                         // bytes per sample
  static constexpr int QS = 16 / EB;                                          // samples per 16 B
  static constexpr int NSEG = AB == 4 ? 2 : 1;                              // output segments per lane
  static constexpr int TT = 32 * S * NSEG;                                    // outputs per tile
  static constexpr int L = (S + OMAX + 1 + QS - 1) / QS * QS;                 // window samples
  static constexpr int LR = L * EB / 4;                                       // window registers
  // largest in-row offset of a warp's last trial past its first (the quad
  // schemes: three steps of at most OMAX + 1)
  static constexpr int OSPAN = AB >= 3 ? 3 * (OMAX + 1) : OMAX;
  static constexpr int ROW = (TT + kMaxOverhang + OSPAN + 2 * QS + 63) / 64 * 64;  // staged samples
  static constexpr int ROWB = ROW * EB;
  static constexpr int THREADS = (NCONS + (ROT ? 0 : 1)) * 32;               // + one producer warp
  static constexpr int DW = NCONS * K <= 32 ? 32 : 64;                        // delays staged per channel
  // two CTAs per SM without a producer warp: one stage buffer fewer, so that
  // both fit the SM's shared memory
  static constexpr int STAGES = MODE == kModeU8 && AB == 1 ? kStagesU8
                                : ALGO == 12                ? 8
                                : ROT                       ? (MINB >= 2 ? kStagesRot - 1 : kStagesRot)
                                                            : kStages;
  static constexpr size_t data_bytes = (size_t)STAGES * kNC * ROWB;
  static constexpr size_t del_bytes = sizeof(int) * (ROT ? NCONS : kDelRing) * kNC * DW;  // ring, or a slot per warp
  // 8-bit mode: per (stage, consumer warp) K int4 of word offsets (one per
  // channel of the stage) and one int4 of byte shifts; else one int4 per
  // (stage, channel, consumer warp)
  static constexpr size_t info_bytes = MODE == kModeU8 && AB == 1 ? sizeof(int4) * STAGES * NCONS * (K + 1)
                                                                     : sizeof(int4) * STAGES * kNC * NCONS;
  // 8-bit DM quads: the 32-bit sums of every consumer thread, [warp][K S][32]
  static constexpr size_t fold_bytes = MODE == kModeU8 && AB == 3 ? sizeof(int) * NCONS * K * S * 32 : 0;
  static constexpr size_t smem = data_bytes + del_bytes + info_bytes + fold_bytes + 16 * STAGES;
  static_assert(smem <= 227 * 1024, "shared memory per CTA");
  // no bank conflicts: register windows (scheme 0) start an odd number of 16-byte
  // units apart, direct 32-bit loads (scheme 1) an odd number of words apart
  static_assert(AB >= 1 ? ((S * EB / 4) % 2 == 1) : ((S * EB / 16) % 2 == 1), "lane stride");
  static_assert(AB != 2 || (MODE != kModeU8 && K == 2), "DM-pair windows: float data, two trials per warp");
  static_assert(AB < 3 || K == 4, "DM-quad windows: four trials per warp");
  static_assert(AB < 4 || MODE == kModeF32, "paired-add DM quads: FP32 staging");
  static_assert(AB != 5 || S % 2 == 1, "in-lane pairs: S = 2 (S / 2) + 1");
  static_assert(AB == 0 || MODE == kModeF32 || S % 2 == 0, "16-bit direct loads pair samples");
  static_assert(MODE != kModeU8 || AB == 1 || AB == 3, "8-bit data: direct loads or DM quads");
  static_assert(!THREADED || MODE == kModeU8, "stage loop in assembly: 8-bit quads");
};

// Per (stage, channel, consumer warp) the producer writes an int4:
//   x = byte offset of lane 0's window in shared memory,
//   y = byte j: in-window offset of DM j of the warp's group,
//   z = number of 16-byte units of the window the channel needs.

// The beam of work item `item`: the last b with cta_start[b] <= item.
__device__ __forceinline__ int item_beam(const BatchArgs& ba, int item) {
  int lo = 0, hi = ba.nbeams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ba.cta_start[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One work item: a (DM tile, time tile) of one beam, by the whole CTA, with
// its mbarriers freshly initialised.  Each warp returns false when one of its
// waits gave up (after letting its own copies land and recording TP_ETIMEOUT).
template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
__device__ __forceinline__ bool dedisperse_item(const BatchArgs& ba, int item) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  constexpr bool ROT = Sh::ROT;
  constexpr int AB = Sh::AB;  // the consumer scheme
  const int bi = item_beam(ba, item);
  const DedispArgs& a = ba.beams[bi];
  const int local = item - ba.cta_start[bi];
  constexpr int TT = Sh::TT, LR = Sh::LR, ROWB = Sh::ROWB, EB = Sh::EB, QS = Sh::QS;
  static_assert(MODE != kModeU8 || K <= 4, "8-bit shifts of a warp's DMs are packed in one int4");
  static_assert(NCONS * K <= 64, "a producer lane holds at most two DMs of the tile");
  static_assert(OMAX < 256, "offsets are packed in bytes");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int STAGES = Sh::STAGES;
  unsigned char* srow = smem_raw;                                                     // [STAGES][kNC][ROWB]
  constexpr int DW = Sh::DW;
  int* sdel = reinterpret_cast<int*>(smem_raw + Sh::data_bytes);                       // [kDelRing][kNC][DW]
  int4* sinfo = reinterpret_cast<int4*>(smem_raw + Sh::data_bytes + Sh::del_bytes);      // [STAGES][kNC][NCONS]
  int* sfold = reinterpret_cast<int*>(smem_raw + Sh::data_bytes + Sh::del_bytes + Sh::info_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + Sh::data_bytes + Sh::del_bytes + Sh::info_bytes +
                                               Sh::fold_bytes);
  uint64_t* empty = full + STAGES;

  const int tile = local % a.ntiles;
  const int tt = local / a.ntiles;
  const DmTile dt = a.tiles[tile];
  const int64_t t0 = (int64_t)tt * TT;
  const int t0m = (int)(t0 & 15);  // t0 mod 16 (staged rows start on 16-byte units)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchan = a.nchan;
  const int nstage = (nchan + kNC - 1) / kNC;
  const int last = dt.nd - 1;
  const unsigned char* ybytes = static_cast<const unsigned char*>(a.y);

  const int32_t* __restrict__ dT = a.delayT;
  // delays of stage st into `slot`: lane l copies delayT[c][d0 + j] for
  // j = l, l + 32 < nd and the kNC channels of the stage (one cp.async group)
  auto prefetch_to = [&](int st, int* slot) {
#pragma unroll
    for (int ci = 0; ci < kNC; ++ci) {
      const int c = st * kNC + ci;
#pragma unroll
      for (int h = 0; h < DW; h += 32) {
        const bool v = st < nstage && c < nchan && lane + h < dt.nd &&
                       in_bounds((int64_t)c * a.dtpitch + dt.d0 + h + lane, 1, a.delayT_elems, a.status);
        cp_async4(slot + ci * DW + h + lane, v ? dT + (int64_t)c * a.dtpitch + dt.d0 + h + lane : dT, v);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // stage i: the window geometry of its (channel, consumer warp) pairs and
  // the bulk copies of its channels onto full[i % STAGES], from its delays
  // `del` (one warp; the stage's buffer must have been released)
  auto issue_stage = [&](int i, const int* del) {
    const int buf = i % STAGES;
    if constexpr (MODE == kModeU8 && AB == 1) {
      // per (channel, consumer warp, DM of its group): byte offset in the
      // stage's rows of the word holding lane 0's first sample, and that
      // sample's shift inside the word (0 or 16 bits)
      // (lane g = w K + j handles DM g of the tile for every channel)
      for (int g = lane; g < NCONS * K; g += 32) {
        const int w = g / K, j = g % K;
        const int jj = g < last ? g : last;
        int off[kNC];
        unsigned shifts = 0;
#pragma unroll
        for (int ci = 0; ci < kNC; ++ci) {
          const int lo = del[ci * DW];
          const int o = del[ci * DW + jj] - lo + ((t0m + lo) & (QS - 1));  // t0 + delay - row start
          off[ci] = (buf * kNC + ci) * ROWB + (o & ~1) * EB;
          shifts |= (unsigned)((o & 1) * 16) << (8 * ci);
        }
        int4* e = sinfo + (buf * NCONS + w) * (K + 1);
        e[j] = make_int4(off[0], off[1], off[2], off[3]);
        reinterpret_cast<unsigned*>(e + K)[j] = shifts;
      }
    }
    // window geometry of every (channel, consumer warp) pair of the stage
    for (int p = lane; (MODE != kModeU8 || AB == 3) && p < kNC * NCONS; p += 32) {
      const int ci = p / NCONS, w = p % NCONS;
      const int g0 = w * K < last ? w * K : last;
      const int lo = del[ci * DW];
      const int dw = del[ci * DW + g0];
      const int64_t base = (t0 + lo) & ~int64_t(QS - 1);
      const int aw = (int)(t0 + dw - base);
      if constexpr (AB >= 3) {
        // four trials sharing one window (scheme 4: one per output segment,
        // 32 S samples apart): the steps e_j = o_j - o_{j-1}
        // between consecutive trials are m or m + 1 (the planner checks
        // this); block index m * 8 + bits.  Trials past the tile's last DM
        // take step m; their sums are never stored.
        int o[4], nreal = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool real = g0 + j <= last;
          o[j] = real ? del[ci * DW + g0 + j] - dw : 0;
          nreal += real ? 1 : 0;
        }
        int m = 1 << 30;
#pragma unroll
        for (int j = 1; j < 4; ++j)
          if (j < nreal) m = min(m, o[j] - o[j - 1]);
        if (nreal < 2) m = 0;
        m = m < 0 ? 0 : (m > OMAX ? OMAX : m);
        int bits = 0;
#pragma unroll
        for (int j = 1; j < 4; ++j) {
          // out-of-pattern steps are clamped so the branch stays inside its
          // table whatever the delays hold
          const int e = j < nreal ? o[j] - o[j - 1] - m : 0;
          bits |= (e > 0 ? 1 : 0) << (j - 1);
        }
        // 16-bit samples: the window starts on the word holding the first
        // trial's first sample, r half-words before it
        const int r = EB == 2 ? (aw & 1) : 0;
        sinfo[(buf * kNC + ci) * NCONS + w] =
            make_int4((buf * kNC + ci) * ROWB + (aw - r) * EB, (r * (OMAX + 1) + m) * 8 + bits, 0, 0);
        continue;
      } else if constexpr (AB >= 1) {
        // sample offset, in the staged row, of each DM's first output of lane 0
        int o[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int jj = g0 + j <= last ? g0 + j : last;
          o[j] = (int)(t0 + del[ci * DW + jj] - base);
        }
        sinfo[(buf * kNC + ci) * NCONS + w] =
            make_int4((buf * kNC + ci) * ROWB, o[0] | (o[1] << 16), o[2] | (o[3] << 16), 0);
        continue;
      }
      int offs = 0, omax = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int jj = g0 + j <= last ? g0 + j : last;
        int o = (aw & (QS - 1)) + del[ci * DW + jj] - dw;
        // the planner bounds o by OMAX; the clamp keeps the indexed branch
        // inside its table whatever the delays hold
        o = o < 0 ? 0 : (o > OMAX ? OMAX : o);
        offs |= o << (8 * j);
        omax = o > omax ? o : omax;
      }
      sinfo[(buf * kNC + ci) * NCONS + w] =
          make_int4((buf * kNC + ci) * ROWB + (aw & ~(QS - 1)) * EB, offs, (S + omax + QS - 1) / QS, 0);
    }
    // lane ci < kNC copies the stage's channel ci: samples
    // [t0 + lo, t0 + TT + hi + QS) rounded out to 16-byte units
    unsigned nb = 0;
    int64_t src = 0;
    if (lane < kNC && i * kNC + lane < nchan) {
      const int lo = del[lane * DW], hi = del[lane * DW + last];
      const int head = (t0m + lo) & (QS - 1);  // row start = t0 + lo - head
      nb = (unsigned)(((TT + hi - lo + QS + head) * EB + 15) & ~15);
      src = ((int64_t)(i * kNC + lane) * a.ypitch + t0 + lo - head) * EB;
      if constexpr (kDebugBounds) {
        // the copy fits its shared-memory row and stays inside the channel's
        // row of the staged series, and the row holds every DM of the tile
        // (delays non-decreasing over the tile's DMs); else it is skipped
        bool ok = in_bounds(0, nb, ROWB, a.status) &&
                  in_bounds(src - (int64_t)(i * kNC + lane) * a.ypitch * EB, nb, a.ypitch * EB, a.status) &&
                  in_bounds(src, nb, a.y_bytes, a.status);
        for (int j = 0; ok && j <= last; ++j) ok = in_bounds(del[lane * DW + j] - lo, 1, hi - lo + 1, a.status);
        if (!ok) nb = 0;
      }
    }
    const unsigned total = __reduce_add_sync(0xffffffffu, nb);
    if (lane == 0) mbar_arrive_expect_tx(&full[buf], total);
    __syncwarp();
    if (nb) bulk_g2s(srow + (buf * kNC + lane) * ROWB, ybytes + src, nb, &full[buf]);
  };

  if (!ROT && warp == NCONS) {
    // ---------------------------------------------------------------- producer
    // delays in a ring of kDelRing stages, kDelRing - 1 stages ahead of use
    auto prefetch = [&](int st) { prefetch_to(st, sdel + (st % kDelRing) * kNC * DW); };
#pragma unroll
    for (int st = 0; st < kDelRing - 1; ++st) prefetch(st);
    bool ok = true;
    int issued = 0;
    for (int i = 0; i < nstage; ++i) {
      __syncwarp();  // every lane is done with the slot the next prefetch reuses
      prefetch(i + kDelRing - 1);
      asm volatile("cp.async.wait_group %0;" ::"n"(kDelRing - 1) : "memory");
      __syncwarp();
      const int buf = i % STAGES;
      if (i >= STAGES) {
        bool got = false;
        if (lane == 0) got = mbar_wait_bounded(&empty[buf], (unsigned)(((i / STAGES) - 1) & 1), ba.wait_tries);
        if (!__shfl_sync(0xffffffffu, got, 0)) {
          ok = false;
          break;
        }
      }
      issue_stage(i, sdel + (i % kDelRing) * kNC * DW);
      ++issued;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // let every issued copy land before the CTA can exit
    if (lane == 0) {
      for (int k = issued - 1; k >= 0 && k >= issued - STAGES; --k)
        if (!mbar_wait_bounded(&full[k % STAGES], (unsigned)((k / STAGES) & 1))) ok = false;
      if (!ok) atomicExch(a.status, TP_ETIMEOUT);
    }
    return ok;
  }

  // ------------------------------------------------------------------ consumers
  const int g0 = warp * K;                 // first tile-local DM of this warp
  const bool live = g0 < dt.nd;

  float acc[K][S];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[j][s] = 0.f;
  // two-segment DM quads: output s of both segments of DM j, packed
  // (segment 0 in the low word)
  constexpr int NSEG = Sh::NSEG;
  unsigned long long acc2[K][AB == 4 ? S : 1];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int s = 0; s < (AB == 4 ? S : 1); ++s) acc2[j][s] = 0ull;
  // in-lane paired DM quads: outputs s and s + S / 2 of DM j packed in
  // accp[j][s] (low word first), output 2 (S / 2) in acct[j]
  constexpr int PH = AB == 5 ? S / 2 : 1;
  unsigned long long accp[K][PH];
  float acct[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    acct[j] = 0.f;
#pragma unroll
    for (int s = 0; s < PH; ++s) accp[j][s] = 0ull;
  }
  // 8-bit mode: pk[j][m] holds outputs 2m, 2m + 1 of DM j as 16-bit lanes
  // (exact: no lane sum reaches 2^16 within kU8FoldStages stages), folded
  // into the 32-bit sums sum32 every kU8FoldStages stages
  constexpr bool U8D = MODE == kModeU8 && AB == 1;  // 8-bit direct loads
  constexpr bool U8Q = MODE == kModeU8 && AB == 3;  // 8-bit DM quads
  constexpr int PW = U8D ? S / 2 : 1;
  constexpr int S32 = U8D ? S : 1;
  // 8-bit DM quads: qe[j][i] holds outputs 2i, 2i + 1 of DM j, qf[j][i]
  // outputs 2i - 1, 2i (16-bit lanes, low first), folded every kU8FoldStages
  // stages into this thread's 32-bit sums in shared memory
  constexpr int QH = U8Q ? S / 2 : 1;
  unsigned qe[K][QH], qf[K][QH + 1];
  int* myfold = sfold + (size_t)warp * K * S * 32 + lane;  // [j S + s][32]
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int q = 0; q < QH; ++q) qe[j][q] = 0u;
#pragma unroll
    for (int q = 0; q <= QH; ++q) qf[j][q] = 0u;
  }
  if constexpr (U8Q) {
#pragma unroll
    for (int q = 0; q < K * S; ++q) myfold[q * 32] = 0;
  }
  unsigned pk[K][PW];
  int sum32[K][S32];
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int m = 0; m < PW; ++m) pk[j][m] = 0u;
#pragma unroll
    for (int s = 0; s < S32; ++s) sum32[j][s] = 0;
  }
  auto fold = [&]() {
    if constexpr (U8Q) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int q = 0; q < QH; ++q) {
          myfold[(j * S + 2 * q) * 32] += (int)(qe[j][q] & 0xffffu) + (int)(qf[j][q] >> 16);
          myfold[(j * S + 2 * q + 1) * 32] += (int)(qe[j][q] >> 16) + (int)(qf[j][q + 1] & 0xffffu);
        }
#pragma unroll
        for (int q = 0; q < QH; ++q) qe[j][q] = 0u;
#pragma unroll
        for (int q = 0; q <= QH; ++q) qf[j][q] = 0u;
      }
    }
    if constexpr (U8D) {
#pragma unroll
      for (int j = 0; j < K; ++j)
#pragma unroll
        for (int m = 0; m < S / 2; ++m) {
          sum32[j][2 * m] += (int)(pk[j][m] & 0xffffu);
          sum32[j][2 * m + 1] += (int)(pk[j][m] >> 16);
          pk[j][m] = 0u;
        }
    }
  };
  using WT = typename std::conditional<MODE == kModeF32, float, unsigned>::type;
  WT w[AB == 0 ? LR : 4];
#pragma unroll
  for (int q = 0; q < (AB == 0 ? LR : 4); ++q) w[q] = 0;
  // the staged words of the lane's outputs 2m, 2m + 1 for one DM and channel,
  // given lane 0's word offset and the half-word shift of its first sample
  const int lane_bytes = lane * S * EB;
  constexpr int NW = MODE == kModeU8 ? S / 2 + 1 : 1;
  auto load_words = [&](int off, unsigned sh, unsigned (&wv)[NW]) {
    const unsigned* r = reinterpret_cast<const unsigned*>(srow + off + lane_bytes);
#pragma unroll
    for (int k = 0; k < NW; ++k) wv[k] = r[k];
    if (sh) {
#pragma unroll
      for (int k = 0; k + 1 < NW; ++k) wv[k] = __funnelshift_r(wv[k], wv[k + 1], 16u);
    }
  };

  // ALGO 6, 7: this warp issues stages warp, warp + NCONS, ..., each
  // kLookRot stages ahead of its use (the buffer it fills was released
  // STAGES - kLookRot stages before, which leaves the warps that much slack),
  // and prefetches the delays of the next one into its own slot right after
  // issuing the previous one
  int* myslot = sdel + warp * kNC * DW;
  int produced = -1;  // the last stage this warp issued
  auto produce = [&](int j) -> bool {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    const int pbuf = j % STAGES;
    if (j >= STAGES) {
      bool got = false;
      if (lane == 0) got = mbar_wait_bounded(&empty[pbuf], (unsigned)(((j / STAGES) - 1) & 1), ba.wait_tries);
      if (!__shfl_sync(0xffffffffu, got, 0)) return false;
    }
    issue_stage(j, myslot);
    produced = j;
    __syncwarp();  // every lane is done with the slot
    if (j + NCONS < nstage) prefetch_to(j + NCONS, myslot);
    return true;
  };
  // after a failed wait: let the copies this warp issued land, then report
  auto bail = [&]() {
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (lane == 0) {
      for (int k = produced; k >= 0 && k > produced - STAGES; k -= NCONS)
        mbar_wait_bounded(&full[k % STAGES], (unsigned)((k / STAGES) & 1));
      atomicExch(a.status, TP_ETIMEOUT);
    }
  };
  if constexpr (ROT) {
    if (warp < nstage) prefetch_to(warp, myslot);
    static_assert(!ROT || Sh::LOOK < STAGES, "lookahead within the pipeline");
    for (int j = warp; j < Sh::LOOK && j < nstage; j += NCONS)
      if (!produce(j)) {
        bail();
        return false;
      }
  }

  for (int i = 0; i < nstage; ++i) {
    const int buf = i % STAGES;
    if constexpr (ROT) {
      const int j = i + Sh::LOOK;
      if (j < nstage && j % NCONS == warp && !produce(j)) {
        bail();
        return false;
      }
    }
    if (!mbar_wait_bounded(&full[buf], (unsigned)((i / STAGES) & 1), ba.wait_tries)) {
      if constexpr (ROT)
        bail();
      else if (lane == 0)
        atomicExch(a.status, TP_ETIMEOUT);
      return false;
    }
    const int nc = nchan - i * kNC < kNC ? nchan - i * kNC : kNC;
    if constexpr (U8D) {
      // direct loads of each DM's words (a half-word funnel shift for odd
      // offsets); two channels at a time so that each accumulator takes both
      // in one three-input add
      if (live) {
        const int4* e = sinfo + (buf * NCONS + warp) * (K + 1);
        const int4 shv = e[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int4 ad = e[j];
          const unsigned shj = (unsigned)(j == 0 ? shv.x : j == 1 ? shv.y : j == 2 ? shv.z : shv.w);
#pragma unroll
          for (int ci = 0; ci < kNC; ci += 2) {
            if (ci >= nc) break;
            unsigned wa[NW];
            load_words(ci == 0 ? ad.x : ad.z, (shj >> (8 * ci)) & 0xffu, wa);
            if (ci + 1 < nc) {
              unsigned wb[NW];
              load_words(ci == 0 ? ad.y : ad.w, (shj >> (8 * ci + 8)) & 0xffu, wb);
#pragma unroll
              for (int m = 0; m < S / 2; ++m) pk[j][m] = pk[j][m] + wa[m] + wb[m];
            } else {
#pragma unroll
              for (int m = 0; m < S / 2; ++m) pk[j][m] += wa[m];
            }
          }
        }
      }
    } else if (live && AB == 2) {
      if constexpr (AB == 2) {
        // one window per channel for the warp's two trials: S + d samples
        // at the first trial's offset, d = the second trial's extra delay
        const unsigned sbase = smem_u32(srow) + (unsigned)(lane * S * EB);
        for (int ci = 0; ci < nc; ++ci) {
          const int4 inf = sinfo[(buf * kNC + ci) * NCONS + warp];
          const int o0 = inf.y & 0xffff, o1 = (inf.y >> 16) & 0xffff;
          int d = o1 - o0;
          // the planner bounds d by OMAX; the clamp keeps the indexed branch
          // inside its table whatever the delays hold
          d = d < 0 ? 0 : (d > OMAX ? OMAX : d);
          if constexpr (MODE == kModeF32)
            add_pair<S, OMAX>(d, sbase + (unsigned)(inf.x + o0 * 4), acc[0], acc[1]);
          else
            add_pair16<S, OMAX, MODE == kModeBF16 ? 1 : 0>((o0 & 1) * (OMAX + 1) + d,
                                                           sbase + (unsigned)(inf.x + (o0 & ~1) * 2), acc[0], acc[1]);
        }
      }
    } else if (live && AB >= 3) {
      if constexpr (AB >= 3) {
        // one window per channel for the warp's four trials, at the first
        // trial's offset
        // (one call site: the loop stays rolled so the jump table is emitted
        // once)
        const unsigned sbase = smem_u32(srow) + (unsigned)(lane * S * EB);
        if constexpr (Sh::THREADED) {
          add_quad8t<S, OMAX, NCONS, ALGO - 6>(sbase, smem_u32(&sinfo[(buf * kNC) * NCONS + warp]), nc, qe, qf);
        } else {
#pragma unroll 1
        for (int ci = 0; ci < nc; ++ci) {
          const int4 inf = sinfo[(buf * kNC + ci) * NCONS + warp];
          if constexpr (AB == 5)
            add_quadp<S, OMAX>(inf.y, sbase + (unsigned)inf.x, accp, acct);
          else if constexpr (AB == 4)
            add_quad2<S, OMAX>(inf.y, sbase + (unsigned)inf.x, acc2);
          else if constexpr (MODE == kModeF32)
            add_quad<S, OMAX>(inf.y, sbase + (unsigned)inf.x, acc);
          else if constexpr (MODE == kModeU8)
            add_quad8<S, OMAX>(inf.y, sbase + (unsigned)inf.x, qe, qf);
          else
            add_quad16<S, OMAX, MODE == kModeBF16 ? 1 : 0>(inf.y, sbase + (unsigned)inf.x, acc);
        }
        }
      }
    } else if (live && AB == 1) {
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
          if constexpr (AB == 0) {
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
    if constexpr (MODE == kModeU8)
      if (i % kU8FoldStages == kU8FoldStages - 1) fold();
  }

  if constexpr (ROT) asm volatile("cp.async.wait_all;" ::: "memory");

  // epilogue: 16-bit and 8-bit modes accumulated the stored samples x~;
  // subtract the block's sum of bandpass values (exact integers for 8-bit data)
  fold();
  if (!live) return true;
  const bool is_int = a.dtype == TP_U8;
  // output s of DM j in segment seg
  auto outv = [&](int j, int seg, int s) -> float {
    if constexpr (AB == 4) {
      const unsigned long long p = acc2[j][s];
      return __uint_as_float(seg ? (unsigned)(p >> 32) : (unsigned)p);
    } else if constexpr (AB == 5) {
      if (s == 2 * PH) return acct[j];
      const unsigned long long p = accp[j][s < PH ? s : s - PH];
      return __uint_as_float(s < PH ? (unsigned)p : (unsigned)(p >> 32));
    } else {
      return acc[j][s];
    }
  };
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
        const int v = (U8D ? sum32[j][U8D ? s : 0] : U8Q ? myfold[(j * S + s) * 32] : __float2int_rn(outv(j, 0, s))) - bint;
        if (tl + s < a.nout && in_bounds((int64_t)d * a.dpitch + tl + s, 1, a.d_elems, a.status)) {
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
      if (lane == 0 && in_bounds((int64_t)d * a.ntt + tt, 1, (int64_t)a.ndm * a.ntt, a.status))
        static_cast<longlong2*>(a.row_part)[(int64_t)d * a.ntt + tt] = make_longlong2(s1, s2);
    } else {
      float* Drow = static_cast<float*>(a.D) + (int64_t)d * a.dpitch;
      float s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int seg = 0; seg < NSEG; ++seg) {
        const int64_t ts = t0 + (int64_t)seg * 32 * S + (int64_t)lane * S;
        float v[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          v[s] = outv(j, seg, s);
          if constexpr (MODE != kModeF32) v[s] = (v[s] - bhi) - blo;
        }
        if (!in_bounds((int64_t)d * a.dpitch + ts, ts + S <= a.nout ? S : (ts < a.nout ? a.nout - ts : 0),
                       a.d_elems, a.status))
          continue;
        if (S % 4 == 0 && ts + S <= a.nout) {
#pragma unroll
          for (int s = 0; s < (S / 4) * 4; s += 4)
            *reinterpret_cast<float4*>(Drow + ts + s) = make_float4(v[s], v[s + 1], v[s + 2], v[s + 3]);
#pragma unroll
          for (int s = 0; s < S; ++s) {
            s1 += v[s];
            s2 += v[s] * v[s];
          }
        } else {
#pragma unroll
          for (int s = 0; s < S; ++s)
            if (ts + s < a.nout) {
              Drow[ts + s] = v[s];
              s1 += v[s];
              s2 += v[s] * v[s];
            }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (lane == 0 && in_bounds((int64_t)d * a.ntt + tt, 1, (int64_t)a.ndm * a.ntt, a.status))
        static_cast<double2*>(a.row_part)[(int64_t)d * a.ntt + tt] = make_double2((double)s1, (double)s2);
    }
  }
  return true;
}

// Initialises the CTA's stage mbarriers (thread 0; the caller synchronises).
template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
__device__ __forceinline__ void init_stage_barriers(uint64_t* full, uint64_t* empty) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  for (int i = 0; i < Sh::STAGES; ++i) {
    mbar_init(&full[i], 1);
    mbar_init(&empty[i], NCONS);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
__device__ __forceinline__ uint64_t* stage_barriers(unsigned char* smem_raw) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  return reinterpret_cast<uint64_t*>(smem_raw + Sh::data_bytes + Sh::del_bytes + Sh::info_bytes + Sh::fold_bytes);
}

// One CTA per work item (grid = cta_start[nbeams]): CTA b runs item b.  The
// work items of a launch are the (beam, DM tile, time tile) triples of every
// beam of the batch.
template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
__global__ void __launch_bounds__(Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>::THREADS, MINB)
    dedisperse_kernel(BatchArgs ba) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = stage_barriers<K, S, OMAX, NCONS, MODE, ALGO, MINB>(smem_raw);
  uint64_t* empty = full + Sh::STAGES;
  if ((int)blockIdx.x >= ba.cta_start[ba.nbeams]) return;
  if (threadIdx.x == 0) init_stage_barriers<K, S, OMAX, NCONS, MODE, ALGO, MINB>(full, empty);
  __syncthreads();
  dedisperse_item<K, S, OMAX, NCONS, MODE, ALGO, MINB>(ba, blockIdx.x);
}

// A persistent grid of a few CTAs per SM drains the same work items: CTA b
// starts with item b and then takes the next untaken item from a device
// counter (the first free CTA gets the next item, so the items stay in order
// and no SM idles while another has a queue).  Between items the CTA
// synchronises (every copy of the item has landed: each warp waited on every
// stage, or drained its own copies when it gave up) and initialises its
// mbarriers afresh.  After a wait gave up the CTA keeps taking items only to
// record TP_ETIMEOUT for their beams, then stops.  A kernel of its own: the
// item loop's back edge, compiled into the one-item kernel, cost its
// one-beam launch 1.2-1.6 % in the instruction schedule.
template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
__global__ void __launch_bounds__(Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>::THREADS, MINB)
    dedisperse_kernel_persistent(BatchArgs ba) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = stage_barriers<K, S, OMAX, NCONS, MODE, ALGO, MINB>(smem_raw);
  uint64_t* empty = full + Sh::STAGES;
  __shared__ int s_item, s_next, s_fail;
  auto take = [&](int cur) {
    return ba.next_item ? (int)gridDim.x + atomicAdd(ba.next_item, 1) : cur + (int)gridDim.x;
  };
  // the loop state lives in shared memory, so that no register stays live
  // across an item (the item's own code uses nearly all of them)
  if (threadIdx.x == 0) s_item = blockIdx.x;
  for (;;) {
    // the next item is taken before this one runs, so that a CTA on its last
    // item (every CTA of a one-CTA-per-item grid) leaves without waiting
    if (threadIdx.x == 0) {
      init_stage_barriers<K, S, OMAX, NCONS, MODE, ALGO, MINB>(full, empty);
      s_fail = 0;
      s_next = s_item < ba.cta_start[ba.nbeams] ? take(s_item) : s_item;
    }
    __syncthreads();
    if (s_item >= ba.cta_start[ba.nbeams]) return;
    const bool ok = dedisperse_item<K, S, OMAX, NCONS, MODE, ALGO, MINB>(ba, s_item);
    if (s_next >= ba.cta_start[ba.nbeams]) return;
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0)
        for (int rest = s_next; rest < ba.cta_start[ba.nbeams]; rest = take(rest))
          atomicExch(ba.beams[item_beam(ba, rest)].status, TP_ETIMEOUT);
      return;
    }
    if (threadIdx.x == 0) s_item = s_next;
  }
}

// grid_limit < 0: one CTA per item; 0: a persistent grid of as many CTAs as
// fit on the device at once; > 0: at most that many CTAs.  A grid that covers
// every item runs the one-item kernel; a smaller one the persistent kernel
// (whose work-item counter, ba.next_item, the caller has zeroed on this
// stream; without one the CTAs step through the items by the grid size).
template <int K, int S, int OMAX, int NCONS, int MODE, int ALGO, int MINB>
cudaError_t launch_mode(const BatchArgs& ba, int ctas, int grid_limit, cudaStream_t s) {
  using Sh = Shape<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  if (ctas <= 0) return cudaErrorInvalidValue;
  auto k1 = dedisperse_kernel<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  auto kp = dedisperse_kernel_persistent<K, S, OMAX, NCONS, MODE, ALGO, MINB>;
  int grid = ctas;
  cudaError_t e = cudaSuccess;
  if (grid_limit == 0) {
    int dev = 0, nsm = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp, Sh::THREADS, Sh::smem);
    if (e != cudaSuccess) return e;
    grid_limit = (per_sm > 0 ? per_sm : 1) * nsm;
  }
  if (grid_limit > 0 && grid_limit < grid) grid = grid_limit;
  auto k = grid < ctas ? kp : k1;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, Sh::THREADS, Sh::smem, s>>>(ba);
  return cudaGetLastError();
}

template <int K, int S, int OMAX, int NCONS, int FMT, int ALGO, int MINB>
cudaError_t launch_shape(const BatchArgs& ba, int dtype, int ctas, int grid_limit, cudaStream_t s) {
  if constexpr (FMT == 4) {
    return launch_mode<K, S, OMAX, NCONS, kModeF32, ALGO, MINB>(ba, ctas, grid_limit, s);
  } else if constexpr (FMT == 3) {
    return launch_mode<K, S, OMAX, NCONS, kModeU8, ALGO, MINB>(ba, ctas, grid_limit, s);
  } else {
    if (dtype == TP_BF16) return launch_mode<K, S, OMAX, NCONS, kModeBF16, ALGO, MINB>(ba, ctas, grid_limit, s);
    return launch_mode<K, S, OMAX, NCONS, kModeF16, ALGO, MINB>(ba, ctas, grid_limit, s);
  }
}

}  // namespace

// The shapes are instantiated in kDedispParts translation units
// (dedisp_p<n>.cu holds the shapes whose index is n modulo kDedispParts) so
// that they compile in parallel; each unit defines TP_DEDISP_PART before
// including this header.
namespace {

template <int I, int K, int S, int OMAX, int NCONS, int FMT, int ALGO, int MINB>
cudaError_t launch_in_part(const BatchArgs& ba, int dtype, int ctas, int grid_limit, cudaStream_t s) {
  if constexpr (I % kDedispParts == TP_DEDISP_PART)
    return launch_shape<K, S, OMAX, NCONS, FMT, ALGO, MINB>(ba, dtype, ctas, grid_limit, s);
  else
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace tp

#define TP_DEDISP_PART_CASE(i, K, S, O, N, F, A, M) \
  case i: return launch_in_part<i, K, S, O, N, F, A, M>(ba, dtype, ctas, grid_limit, s);

// Defines tp::launch_dedisperse_part<n>: the launches of this unit's shapes.
#define TP_DEFINE_DEDISP_PART(n)                                                                      \
  namespace tp {                                                                                       \
  cudaError_t launch_dedisperse_part##n(int shape, int dtype, const BatchArgs& ba, int ctas,           \
                                        int grid_limit, cudaStream_t s) {                              \
    switch (shape) {                                                                                   \
      TP_SHAPES(TP_DEDISP_PART_CASE)                                                                   \
      default: return cudaErrorInvalidValue;                                                           \
    }                                                                                                  \
  }                                                                                                    \
  }
