// Kernel shapes of the dedispersion kernel (A5, Sec. 2.2.2), shared by the
// shape table and the units that instantiate the kernels.
#pragma once

// Kernel shapes: (DMs per warp K, outputs per lane S, largest in-window offset
// OMAX, consumer warps).  The planner keeps the shapes whose K-trial groups
// all spread by at most OMAX - 3 samples; the autotuner (or the first
// feasible shape) picks among them.
// FMT = staging format: 4 FP32 y (FP32 data), 2 16-bit float x~ (binary16 and
// bfloat16 data), 3 8-bit x~ widened to 16-bit integers.
// ALGO 0: register window + jump-table shifted adds (reuse across the K DMs);
// ALGO 1: direct shared loads per DM (no offset bound, OMAX unused);
// ALGO 2: DM pairs sharing one window, second trial's extra delay <= OMAX;
// ALGO 3: DM quads sharing one window, steps between consecutive trials m or
// m + 1 with m <= OMAX;
// ALGO 4: ALGO 3 over two output segments per lane (32 S samples apart), both
// added by one paired FP32 add (FP32 staging only);
// ALGO 5: ALGO 3 with the lane's outputs s and s + S / 2 added by one paired
// FP32 add (S odd; FP32 staging only);
// ALGO 6, 7, 8: ALGO 4, 5, 3 without a producer warp: all NCONS warps consume,
// and warp w also issues the copies of stages w, w + NCONS, ...;
// ALGO 9: ALGO 8 (8-bit data) with threaded dispatch over a stage's channels.
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
  X(16, 2, 22, 0, 16, 2, 1, 1)        \
  X(17, 2, 18, 0, 8, 3, 1, 2)        \
  X(18, 2, 26, 0, 15, 3, 1, 1)       \
  X(19, 1, 38, 0, 15, 3, 1, 1)       \
  X(20, 4, 18, 0, 8, 3, 1, 1)        \
  X(21, 2, 34, 0, 8, 3, 1, 1)        \
  X(22, 1, 42, 0, 15, 3, 1, 1)       \
  X(23, 3, 26, 0, 10, 3, 1, 1)       \
  X(24, 2, 25, 11, 15, 4, 2, 1)      \
  X(25, 2, 25, 11, 8, 4, 2, 2)       \
  X(26, 2, 21, 15, 8, 4, 2, 2)       \
  X(27, 2, 29, 11, 15, 4, 2, 1)      \
  X(28, 2, 26, 11, 15, 2, 2, 1)      \
  X(29, 2, 22, 11, 8, 2, 2, 2)        \
  X(30, 4, 25, 9, 8, 4, 3, 1)        \
  X(31, 4, 31, 9, 8, 4, 3, 1)        \
  X(32, 4, 23, 9, 8, 4, 3, 1)        \
  X(33, 4, 31, 9, 11, 4, 3, 1)       \
  X(34, 4, 25, 9, 11, 4, 3, 1)       \
  X(35, 4, 25, 9, 15, 4, 3, 1)       \
  X(36, 4, 26, 9, 8, 2, 3, 1)        \
  X(37, 4, 26, 9, 11, 2, 3, 1)       \
  X(38, 4, 30, 9, 11, 2, 3, 1)       \
  X(39, 4, 26, 16, 7, 3, 3, 1)       \
  X(40, 4, 18, 16, 11, 3, 3, 1)      \
  X(41, 4, 22, 16, 7, 3, 3, 1)        \
  X(42, 4, 41, 9, 7, 4, 3, 1)        \
  X(43, 4, 30, 16, 7, 3, 3, 1)      \
  X(44, 4, 15, 9, 11, 4, 4, 1)       \
  X(45, 4, 21, 9, 7, 4, 4, 1)        \
  X(46, 4, 23, 9, 7, 4, 4, 1)        \
  X(47, 4, 19, 9, 7, 4, 4, 1)        \
  X(48, 4, 45, 9, 7, 4, 5, 1)        \
  X(49, 4, 43, 9, 7, 4, 5, 1)        \
  X(50, 4, 27, 9, 11, 4, 5, 1)       \
  X(51, 4, 25, 9, 11, 4, 5, 1)       \
  X(52, 4, 29, 9, 11, 4, 5, 1)       \
  X(53, 4, 23, 9, 8, 4, 6, 1)        \
  X(54, 4, 29, 9, 12, 4, 7, 1)       \
  X(55, 4, 45, 9, 8, 4, 7, 1)        \
  X(56, 4, 21, 9, 8, 4, 6, 1)        \
  X(57, 4, 30, 16, 8, 3, 8, 1)       \
  X(58, 4, 26, 16, 8, 3, 8, 1)       \
  X(59, 4, 30, 16, 8, 3, 9, 1)       \
  X(60, 4, 26, 16, 8, 3, 9, 1)       \
  X(61, 4, 22, 16, 8, 3, 9, 1)       \
  X(62, 4, 30, 16, 8, 3, 10, 1)      \
  X(63, 4, 30, 16, 8, 3, 11, 1)      \
  X(64, 4, 14, 16, 8, 3, 8, 2)       \
  X(65, 4, 14, 16, 8, 3, 10, 2)      \
  X(66, 4, 26, 16, 8, 3, 12, 1)      \
  X(67, 4, 22, 16, 8, 3, 12, 1)

namespace tp {
constexpr int kDedispParts = 12;  // translation units the kernel instantiations are split over
}  // namespace tp
