// Launchers of the factored OLS beta refresh (lv_ols.cu); the other OLS
// launchers are declared with the rest of the library's in lv_internal.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lv {

// beta (row-major n x p, ld) += (G_1 - G_2) Y_R + G H with H = Wu^T C
// (2k x p, computed into H first); G, Wu, C column-major with column stride
// fs (G and Wu n x 2k, C n x p), Y_R k x p row-major.
template <typename T>
cudaError_t launch_beta_update(T* beta, int64_t ld, const T* G, const T* Wu, const T* Cc,
                               int64_t fs, int n, int p, int k, const T* Yr, T* H,
                               cudaStream_t s);

}  // namespace lv
