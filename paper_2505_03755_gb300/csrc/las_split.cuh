// Split-precision (BF16 digit) path: emulated-FP64 GEMMs on tcgen05 tensor cores.
#pragma once
#include "las_common.cuh"

struct SplitState;

las_status split_create(SplitState** s, int n, int X, int op, int Lc, const double* Bp,
                        cudaStream_t st, size_t* bytes);
void split_destroy(SplitState* s);
las_status split_prepare_C(SplitState* s, const double* Cocc, cudaStream_t st);
las_status split_half_full(SplitState* s, int l0, int nL, const double* Cocc, double* Ht,
                           double* T, cudaStream_t st);
las_status split_project(SplitState* s, int nL, const double* Ht, const double* W, double* Out,
                         int accumulate, cudaStream_t st);
