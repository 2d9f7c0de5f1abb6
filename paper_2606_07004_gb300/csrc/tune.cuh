// Autotuner of the Krylov step kernels' layout (see tune.cu).
#pragma once

#include "krylov.cuh"

namespace ld {

// The fastest TuneCfg for a matrix and block width, timed once and cached.
template <typename T>
int autotune_krylov(const int* rowptr, const int* colind, const typename ValOf<T>::type* vals, int n,
                    long long nnz, int ld, int ndots, int nbasis, int extra, cudaStream_t st,
                    TuneCfg* out);

}  // namespace ld
