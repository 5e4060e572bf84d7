// Seeded N(0,1) start blocks (Philox4x32-10 + Box-Muller; definition in rng.cu).
#pragma once
#include <cuda_runtime.h>

namespace mpl {

// X (n x m column-major, real doubles or interleaved complex) <- the block
// drawn for ``seed``; complex entries are (z0 + i z1) / sqrt 2.
void start_block(cudaStream_t st, bool cx, long long n, int m, unsigned long long seed, double* X);

}  // namespace mpl
