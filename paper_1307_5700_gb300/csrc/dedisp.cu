// A5: the dedispersion kernel's shape table and launch dispatch (Sec. 2.2.2).
// The kernel itself is in dedisp_kernel.cuh, instantiated per shape in
// dedisp_p0.cu .. dedisp_p11.cu.
#include "dedisp_shapes.cuh"
#include "tp_common.cuh"

namespace tp {

cudaError_t launch_dedisperse_part0(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part1(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part2(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part3(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part4(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part5(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part6(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part7(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part8(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part9(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_part10(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                       cudaStream_t s);
cudaError_t launch_dedisperse_part11(int shape, int dtype, const BatchArgs& ba, int ctas, int grid_limit,
                                       cudaStream_t s);
static_assert(kDedispParts == 12, "one launch_dedisperse_part per unit");

#define TP_SHAPE_ENTRY(i, K, S, O, N, F, A, M) {K, S, O, N, F, A},
const KernelShape kShapes[kNumShapes] = {TP_SHAPES(TP_SHAPE_ENTRY)};
#undef TP_SHAPE_ENTRY

int shape_tile_t(int shape) {
  const int algo = kShapes[shape].ALGO;
  return (algo == 4 || algo == 6 ? 64 : 32) * kShapes[shape].S;  // two output segments per lane
}

cudaError_t launch_dedisperse(int shape, int dtype, const BatchArgs& ba, int ctas, cudaStream_t s, int grid_limit) {
  if (shape < 0 || shape >= kNumShapes) return cudaErrorInvalidValue;
  switch (shape % kDedispParts) {
    case 0: return launch_dedisperse_part0(shape, dtype, ba, ctas, grid_limit, s);
    case 1: return launch_dedisperse_part1(shape, dtype, ba, ctas, grid_limit, s);
    case 2: return launch_dedisperse_part2(shape, dtype, ba, ctas, grid_limit, s);
    case 3: return launch_dedisperse_part3(shape, dtype, ba, ctas, grid_limit, s);
    case 4: return launch_dedisperse_part4(shape, dtype, ba, ctas, grid_limit, s);
    case 5: return launch_dedisperse_part5(shape, dtype, ba, ctas, grid_limit, s);
    case 6: return launch_dedisperse_part6(shape, dtype, ba, ctas, grid_limit, s);
    case 7: return launch_dedisperse_part7(shape, dtype, ba, ctas, grid_limit, s);
    case 8: return launch_dedisperse_part8(shape, dtype, ba, ctas, grid_limit, s);
    case 9: return launch_dedisperse_part9(shape, dtype, ba, ctas, grid_limit, s);
    case 10: return launch_dedisperse_part10(shape, dtype, ba, ctas, grid_limit, s);
    default: return launch_dedisperse_part11(shape, dtype, ba, ctas, grid_limit, s);
  }
}

}  // namespace tp
