// Shared host/device utilities of liblogdet: error plumbing, the SplitMix64
// probe generator, vector load/store helpers and compensated FP32 sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>

#include "../../include/logdet.h"

namespace ld {

// ---------------------------------------------------------------------------
// Errors.  Every host function returns an int code; the detail text of the
// calling thread's last failure is kept in a thread-local string.
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
const char* last_error();

#define LD_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      ::ld::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,              \
                      cudaGetErrorString(e_));                                 \
      return e_ == cudaErrorMemoryAllocation ? LOGDET_ENOMEM : LOGDET_ECUDA;   \
    }                                                                          \
  } while (0)

#define LD_TRY(expr)                                                           \
  do {                                                                         \
    int rc_ = (expr);                                                          \
    if (rc_ != LOGDET_OK) return rc_;                                          \
  } while (0)

#define LD_CHECK_LAUNCH() LD_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood 2014): output finaliser and the probe
// entry of (seed, stream, col, row) as defined in logdet.h.
// ---------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t probe_key(uint64_t seed, int stream) {
  return sm64_mix(seed + (uint64_t)(stream + 1) * kGolden);
}

// +1 or -1 for entry (row, col) of the stream whose key is `key`.
__host__ __device__ __forceinline__ int probe_sign(uint64_t key, uint32_t col, uint32_t row) {
  uint64_t ctr = ((uint64_t)col << 32) + (uint64_t)row + 1ull;
  return (sm64_mix(key + ctr * kGolden) >> 63) ? -1 : 1;
}

// Standard normal entry (row, col) from the same counter (Box-Muller): with z
// the counter output and w = mix(z), u1 = ((z >> 11) + 1) 2^-53 in (0, 1],
// u2 = (w >> 11) 2^-53 in [0, 1), g = sqrt(-2 log u1) cos(2 pi u2).
__device__ __forceinline__ double probe_gauss(uint64_t key, uint32_t col, uint32_t row) {
  const uint64_t ctr = ((uint64_t)col << 32) + (uint64_t)row + 1ull;
  const uint64_t z = sm64_mix(key + ctr * kGolden);
  const uint64_t w = sm64_mix(z);
  const double u1 = ((double)(z >> 11) + 1.0) * 0x1p-53;
  const double u2 = (double)(w >> 11) * 0x1p-53;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

__device__ __forceinline__ double probe_value(uint64_t key, uint32_t col, uint32_t row, int gaussian) {
  return gaussian ? probe_gauss(key, col, row) : (double)probe_sign(key, col, row);
}

// ---------------------------------------------------------------------------
// 16-byte vectors of the block element type.
// ---------------------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };
template <> struct Vec16<float>  { using type = float4;  static constexpr int N = 4; };

template <typename T>
__device__ __forceinline__ void load_vec(const T* p, T (&v)[Vec16<T>::N]) {
  using V = typename Vec16<T>::type;
  V t = __ldg(reinterpret_cast<const V*>(p));
  if constexpr (Vec16<T>::N == 2) { v[0] = t.x; v[1] = t.y; }
  else { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
}

// Plain (coherent) load for data written earlier in the same kernel chain.
template <typename T>
__device__ __forceinline__ void load_vec_cg(const T* p, T (&v)[Vec16<T>::N]) {
  using V = typename Vec16<T>::type;
  V t = *reinterpret_cast<const V*>(p);
  if constexpr (Vec16<T>::N == 2) { v[0] = t.x; v[1] = t.y; }
  else { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
}

template <typename T>
__device__ __forceinline__ void store_vec(T* p, const T (&v)[Vec16<T>::N]) {
  using V = typename Vec16<T>::type;
  V t;
  if constexpr (Vec16<T>::N == 2) { t.x = v[0]; t.y = v[1]; }
  else { t.x = v[0]; t.y = v[1]; t.z = v[2]; t.w = v[3]; }
  *reinterpret_cast<V*>(p) = t;
}

// ---------------------------------------------------------------------------
// Dot-product accumulators.  FP64 blocks accumulate with FMA in FP64.  FP32
// blocks use a compensated dot (the product's rounding error from an FMA plus
// a TwoSum of the running sum: Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, Algorithm Dot2), all in FP32.
// ---------------------------------------------------------------------------
struct AccD {
  double s;
  __device__ __forceinline__ void zero() { s = 0.0; }
  __device__ __forceinline__ void fma(double a, double b) { s = ::fma(a, b, s); }
  __device__ __forceinline__ void add(const AccD& o) { s += o.s; }
  __device__ __forceinline__ double value() const { return s; }
};

struct AccF {
  float s, e;
  __device__ __forceinline__ void zero() { s = 0.f; e = 0.f; }
  // The _rn intrinsics are never contracted into FMAs, which TwoSum needs.
  __device__ __forceinline__ void two_sum_into(float x) {
    float t = __fadd_rn(s, x);
    float bp = __fsub_rn(t, s);
    float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    e = __fadd_rn(e, err);
  }
  __device__ __forceinline__ void fma(float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = __fmaf_rn(a, b, -p);
    two_sum_into(p);
    e = __fadd_rn(e, pe);
  }
  __device__ __forceinline__ void add(const AccF& o) {
    two_sum_into(o.s);
    e = __fadd_rn(e, o.e);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

template <typename T> struct AccOf;
template <> struct AccOf<double> { using type = AccD; };
template <> struct AccOf<float>  { using type = AccF; };

// Partial sums written by the block kernels and reduced by the scalar kernels.
// FP64 blocks store one double per partial; FP32 blocks store the (s, e) pair.
template <typename T> struct PartOf;
template <> struct PartOf<double> { using type = double; };
template <> struct PartOf<float>  { using type = float2; };

__device__ __forceinline__ void put_part(double* p, const AccD& a) { *p = a.s; }
__device__ __forceinline__ void put_part(float2* p, const AccF& a) { *p = make_float2(a.s, a.e); }
__device__ __forceinline__ void get_part(const double* p, AccD& a) { a.s = *p; }
__device__ __forceinline__ void get_part(const float2* p, AccF& a) { float2 t = *p; a.s = t.x; a.e = t.y; }

__host__ __device__ __forceinline__ int div_up(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int round_up(int a, int b) { return div_up(a, b) * b; }

}  // namespace ld
