#include "las_split.cuh"

struct SplitState { int dummy; };

las_status split_create(SplitState** s, int, int, int, int, const double*, cudaStream_t, size_t*) {
  *s = nullptr;
  return LAS_ERR_UNSUPPORTED;
}
void split_destroy(SplitState*) {}
las_status split_prepare_C(SplitState*, const double*, cudaStream_t) { return LAS_ERR_UNSUPPORTED; }
las_status split_half_full(SplitState*, int, int, const double*, double*, double*, cudaStream_t) {
  return LAS_ERR_UNSUPPORTED;
}
las_status split_project(SplitState*, int, const double*, const double*, double*, int, cudaStream_t) {
  return LAS_ERR_UNSUPPORTED;
}
