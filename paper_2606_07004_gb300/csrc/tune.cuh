// Autotuner of the Krylov step kernels' layout (see tune.cu).
#pragma once

#include "handle.cuh"
#include "krylov.cuh"

namespace ld {

// The fastest TuneCfg for a matrix and block width, timed once and cached.
// vals: the solve's scaled values of h's matrix.
template <typename T>
int autotune_krylov(logdet_ctx* h, const typename ValOf<T>::type* vals, int ld, int ndots,
                    int nbasis, int extra, cudaStream_t st, TuneCfg* out);

}  // namespace ld
