// Matrix-free gridded operators: Q acts on fields on an nx x ny grid (row
// index y * nx + x) as
//   Q[(y, x), (y', x')] = W(|y - y'|, |x - x'|)   for |y - y'|, |x - x'| <= R,
// and 0 otherwise (a compactly supported stationary covariance restricted to
// the grid, e.g. the Wendland covariance of the paper's GRF study, Sec. 4).
// W is a quadrant table of (R + 1)^2 values.  The operator is applied by a
// register-tiled convolution over shared-memory rows; nothing of size
// n x (stencil) is stored.
#pragma once

#include "handle.cuh"

namespace ld {

constexpr int kMaxGridRadius = 96;
constexpr int kGridP = 8;          // outputs per thread along x
constexpr int kGridTX = 32;        // threads along x: an x segment of 256 outputs
constexpr int kGridTY = 8;         // output rows per CTA (one warp each)
constexpr int kGridThreads = kGridTX * kGridTY;

// Row length of the expanded table: W(dy, dx) at [dy * L + dx + R], dx in
// [-R, R], followed by kGridP zeros.
inline int grid_row_len(int R) { return 2 * R + 1 + kGridP; }

int create_grid_handle(int nx, int ny, int R, const double* w, logdet_handle* out);

// Expanded table of W / c in the compute type CT (double or float).
template <typename CT>
int grid_table(const logdet_ctx* h, double c, CT* out, cudaStream_t st);
size_t grid_table_count(const logdet_ctx* h);

// y = Q x (+ colshift[p] x[:, p]) on a block (n x ld), tab from grid_table.
template <typename T>
int grid_apply(const logdet_ctx* h, const typename Compute<T>::type* tab, const T* x, T* y,
               int ld, const double* colshift, cudaStream_t st);

// Partials [d][ld][ntiles] of dotv_d . y over uniform tiles (the pass-1
// dots of a Krylov step whose SpMM is grid_apply).
template <typename T>
int dots_pass(const T* y, const T* const* dotv, int ndots, typename PartOf<T>::type* part, int n,
              int ld, int tile_rows, int ntiles, int threads, cudaStream_t st);

}  // namespace ld
