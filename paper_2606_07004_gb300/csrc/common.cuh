// Shared host/device utilities of liblogdet: error plumbing, the SplitMix64
// probe generator, vector load/store helpers and compensated FP32 sums.
#pragma once

#include <cuda_bf16.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>
#include <type_traits>

#include "../../include/logdet.h"

namespace ld {

// Grid structure of a stencil matrix: every entry lies on one of a few
// diagonals.  dim 2: each diagonal offset is line * L + c with a line
// stride L, lines in [-A, A] and small c (a 2D grid stencil: L = the grid's
// row length).  dim 3: the matrix is a stencil on an L x ny x nz grid (row
// = (z * ny + y) * L + x) with offsets dz * P + dy * L + dx (P = L ny),
// |dz| <= A, |dy| <= Ay, |dx| <= Ax, and no entry wrapping across a line or
// plane edge.  See dia.cu.
constexpr int kMaxDiags = 16;
struct DiaInfo {
  int ndiag;                  // 0: no such structure
  int dim;                    // 2 or 3
  int off[kMaxDiags];         // ascending
  int L;                      // line stride
  int A;                      // lines (dim 2) or planes (dim 3) -A .. A
  int cmin, cw;               // dim 2: c ranges over [cmin, cmin + cw]
  int line[kMaxDiags];        // line (dim 2) or plane (dim 3) offset of each diagonal
  int cpos[kMaxDiags];        // dim 2: c - cmin of each diagonal
  int P, ny, nz, Ay, Ax;      // dim 3: plane stride, grid lines per plane, planes, radii
  int dy[kMaxDiags], dx[kMaxDiags];  // dim 3: in-plane offsets of each diagonal
};


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
// Block element types.  A block stores T; arithmetic runs in Compute<T>
// (BF16 vectors compute in FP32); matrix values are ValOf<T> (FP32 for BF16
// vectors).  One vector load brings Vec16<T>::N elements: 16 bytes for FP64
// and FP32, 8 bytes (four elements) for BF16, so that a thread holds as many
// compensated FP32 accumulators for a BF16 block as for an FP32 one.
// ---------------------------------------------------------------------------
using bf16 = __nv_bfloat16;

// Double-float vectors (LOGDET_MIXED_F32X2): each entry is stored as the
// unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2 (about 48
// significand bits in 8 bytes), and computed on in dfloat arithmetic built
// from error-free transformations on the FP32 pipe (Knuth's TwoSum, the
// FMA TwoProduct; the double-double algorithms of Hida, Li and Bailey 2001
// at single precision).  The _rn intrinsics keep the compiler from
// contracting the error terms into FMAs.
struct f32x2 {
  float hi, lo;
};
// dfloat and its operators live in a namespace of their own: found by
// argument-dependent lookup for dfloat operands, they do not hide ::fma
// from unqualified calls on doubles and floats elsewhere in ld.
namespace dfl {
struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(float h) : hi(h), lo(0.f) {}
  __host__ __device__ constexpr dfloat(int i) : hi((float)i), lo(0.f) {}
  __host__ __device__ explicit dfloat(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ dfloat df_renorm(float s, float e) {  // quick TwoSum, |s| >= |e|
  const float t = __fadd_rn(s, e);
  return dfloat(t, __fsub_rn(e, __fsub_rn(t, s)));
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_renorm(s, e);
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_renorm(p, e);
}
// a b + c: the unnormalised TwoProduct of a b (with both cross terms) fed
// straight into the TwoSum with c, one renormalisation at the end.
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  return df_renorm(s, e);
}
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, -b); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = df_add(a, b); }
}  // namespace dfl
using dfl::dfloat;

template <typename T> struct Compute { using type = T; };
template <> struct Compute<bf16> { using type = float; };
template <> struct Compute<f32x2> { using type = dfloat; };
template <typename T> struct ValOf { using type = T; };
template <> struct ValOf<bf16> { using type = float; };
template <> struct ValOf<f32x2> { using type = float; };

template <typename T> struct Vec16;
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };
template <> struct Vec16<float>  { using type = float4;  static constexpr int N = 4; };
template <> struct Vec16<bf16>   { using type = uint2;   static constexpr int N = 4; };
template <> struct Vec16<f32x2>  { using type = float4;  static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ void load_vec(const T* p, typename Compute<T>::type (&v)[Vec16<T>::N]) {
  using V = typename Vec16<T>::type;
  V t = __ldg(reinterpret_cast<const V*>(p));
  if constexpr (std::is_same<T, double>::value) { v[0] = t.x; v[1] = t.y; }
  else if constexpr (std::is_same<T, float>::value) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
  else if constexpr (std::is_same<T, f32x2>::value) { v[0] = dfloat(t.x, t.y); v[1] = dfloat(t.z, t.w); }
  else {
    const uint32_t w[2] = {t.x, t.y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
      float2 f = __bfloat1622float2(h2);
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_vec(T* p, const typename Compute<T>::type (&v)[Vec16<T>::N]) {
  using V = typename Vec16<T>::type;
  V t;
  if constexpr (std::is_same<T, double>::value) { t.x = v[0]; t.y = v[1]; }
  else if constexpr (std::is_same<T, float>::value) { t.x = v[0]; t.y = v[1]; t.z = v[2]; t.w = v[3]; }
  else if constexpr (std::is_same<T, f32x2>::value) {
    t.x = v[0].hi; t.y = v[0].lo; t.z = v[1].hi; t.w = v[1].lo;
  }
  else {
    uint32_t w[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    t.x = w[0]; t.y = w[1];
  }
  *reinterpret_cast<V*>(p) = t;
}

// Scalar conversions between block element types (BF16 via FP32, round to nearest).
template <typename To, typename From>
__host__ __device__ __forceinline__ To cvt(From x) {
  if constexpr (std::is_same<To, bf16>::value) return __float2bfloat16_rn((float)x);
  else if constexpr (std::is_same<From, bf16>::value) return (To)__bfloat162float(x);
  else if constexpr (std::is_same<To, f32x2>::value) {
    const dfloat d((double)x);
    return f32x2{d.hi, d.lo};
  } else if constexpr (std::is_same<From, f32x2>::value) return (To)((double)x.hi + (double)x.lo);
  else return (To)x;
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

// Two compensated FP32 accumulators in packed pairs (Blackwell's
// add/sub/mul/fma .rn.f32x2: two IEEE single-precision operations per
// instruction, each lane rounded exactly as the scalar _rn intrinsic).  Lane
// i performs exactly the operations of an AccF in the same order, so
// lo()/hi() equal what two AccF would hold; the instruction count halves.
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
struct AccF2 {
  unsigned long long s, e;
  __device__ __forceinline__ void zero() { s = 0ull; e = 0ull; }
  // s + e += a * b per lane: TwoProduct (product and its FMA error), TwoSum.
  __device__ __forceinline__ void fma(unsigned long long a, unsigned long long b) {
    const unsigned long long p = f2_mul(a, b);
    const unsigned long long pe = f2_fma(a, b, p ^ 0x8000000080000000ull);  // a b - p
    const unsigned long long t = f2_add(s, p);
    const unsigned long long bp = f2_sub(t, s);
    const unsigned long long err = f2_add(f2_sub(s, f2_sub(t, bp)), f2_sub(p, bp));
    s = t;
    e = f2_add(e, err);
    e = f2_add(e, pe);
  }
  __device__ __forceinline__ AccF lo() const {
    AccF r;
    float sh, eh;
    f2_unpack(s, r.s, sh);
    f2_unpack(e, r.e, eh);
    return r;
  }
  __device__ __forceinline__ AccF hi() const {
    AccF r;
    float sl, el;
    f2_unpack(s, sl, r.s);
    f2_unpack(e, el, r.e);
    return r;
  }
};

template <typename T> struct AccOf;
template <> struct AccOf<double> { using type = AccD; };
template <> struct AccOf<float>  { using type = AccF; };
template <> struct AccOf<bf16>   { using type = AccF; };

// Partial sums written by the block kernels and reduced by the scalar kernels.
// FP64 blocks store one double per partial; FP32 blocks store the (s, e) pair.
template <typename T> struct PartOf;
template <> struct PartOf<double> { using type = double; };
template <> struct PartOf<float>  { using type = float2; };
template <> struct PartOf<bf16>   { using type = float2; };

// Double-float blocks: a compensated FP32 sum of hi * hi (as AccF) with the
// cross terms hi * lo + lo * hi added to its error word; partials as AccF's.
struct AccDF {
  AccF a;
  __device__ __forceinline__ void zero() { a.zero(); }
  __device__ __forceinline__ void fma(dfloat u, dfloat y) {
    a.fma(u.hi, y.hi);
    a.e = __fadd_rn(a.e, __fmaf_rn(u.hi, y.lo, __fmul_rn(u.lo, y.hi)));
  }
  __device__ __forceinline__ void add(const AccDF& o) { a.add(o.a); }
  __device__ __forceinline__ double value() const { return a.value(); }
};
template <> struct AccOf<f32x2> { using type = AccDF; };
template <> struct PartOf<f32x2> { using type = float2; };
__device__ __forceinline__ void put_part(float2* p, const AccDF& a) { *p = make_float2(a.a.s, a.a.e); }
__device__ __forceinline__ void get_part(const float2* p, AccDF& a) { float2 t = *p; a.a.s = t.x; a.a.e = t.y; }

__device__ __forceinline__ void put_part(double* p, const AccD& a) { *p = a.s; }
__device__ __forceinline__ void put_part(float2* p, const AccF& a) { *p = make_float2(a.s, a.e); }
__device__ __forceinline__ void get_part(const double* p, AccD& a) { a.s = *p; }
__device__ __forceinline__ void get_part(const float2* p, AccF& a) { float2 t = *p; a.s = t.x; a.e = t.y; }

__host__ __device__ __forceinline__ int div_up(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int round_up(int a, int b) { return div_up(a, b) * b; }

}  // namespace ld
