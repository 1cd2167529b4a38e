// common.cuh -- shared device helpers for the qwb kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/qwb.h"

namespace qwb {

// ---- error plumbing (host) ------------------------------------------------
void set_last_error(const std::string& msg);
void count_launch(int64_t k = 1);
int cuda_fail(cudaError_t e, const char* what);

#define QWB_CUDA(call)                                         \
    do {                                                       \
        cudaError_t qwb_e_ = (call);                           \
        if (qwb_e_ != cudaSuccess) return cuda_fail(qwb_e_, #call); \
    } while (0)

// Check a kernel launch and count it.
#define QWB_LAUNCHED()                                         \
    do {                                                       \
        count_launch();                                        \
        cudaError_t qwb_e_ = cudaGetLastError();               \
        if (qwb_e_ != cudaSuccess) return cuda_fail(qwb_e_, "kernel launch"); \
    } while (0)

// ---- directed rounding, overloaded on the scalar type ----------------------
// rd = toward -infinity, ru = toward +infinity (IEEE-correct intrinsics).
__device__ __forceinline__ float sub_rd(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ double sub_rd(double a, double b) { return __dsub_rd(a, b); }
__device__ __forceinline__ float add_ru(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ double add_ru(double a, double b) { return __dadd_ru(a, b); }
__device__ __forceinline__ float fma_ru(float a, float b, float c) { return __fmaf_ru(a, b, c); }
__device__ __forceinline__ double fma_ru(double a, double b, double c) { return __fma_ru(a, b, c); }
__device__ __forceinline__ float mul_ru(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ double mul_ru(double a, double b) { return __dmul_ru(a, b); }

template <typename T> __device__ __forceinline__ T from_double_ru(double x);
template <> __device__ __forceinline__ float from_double_ru<float>(double x) { return __double2float_ru(x); }
template <> __device__ __forceinline__ double from_double_ru<double>(double x) { return x; }
template <typename T> __device__ __forceinline__ T from_double_rn(double x);
template <> __device__ __forceinline__ float from_double_rn<float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ double from_double_rn<double>(double x) { return x; }

// FP32 -> FP64 widening by exponent re-biasing on the integer pipes, exact
// for every float (normal, subnormal, zero, infinity, NaN), which keeps bulk
// widening off the FP64 pipe.
__device__ __forceinline__ double widen_f32(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    unsigned long long ebits;
    if (e == 0xffu) {
        ebits = 0x7ffull;                       // infinity or NaN (payload kept)
    } else if (e != 0u) {
        ebits = e + 896u;                       // 1023 - 127
    } else if (m == 0u) {
        ebits = 0ull;                           // signed zero
    } else {                                    // subnormal m * 2^-149: normalise
        const int sh = __clz(m) - 8;            // brings the leading one to bit 23
        m = (m << sh) & 0x7fffffu;
        ebits = (unsigned long long)(897 - sh);
    }
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | (ebits << 52) |
                                    ((unsigned long long)m << 29);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen_f32(double v) { return v; }
// The same for a value that is usually a positive normal float (a C-bar
// entry): then the FP64 bits are the FP32 bits shifted by 29 with the
// exponent re-biased by 1023 - 127; anything else takes widen_f32.
__device__ __forceinline__ double widen_pos_f32(float v) {
    const unsigned u = __float_as_uint(v);
    if (u - 0x00800000u < 0x7f000000u)                  // sign 0, exponent field 1..254
        return __longlong_as_double((long long)(((unsigned long long)u << 29) + (896ull << 52)));
    return widen_f32(v);
}

template <typename T> __device__ __forceinline__ T pos_inf();
template <> __device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double pos_inf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

// Atomic minimum on a float/double stored as such.  Values with a clear sign
// bit order like signed integers, values with the sign bit set order in
// reverse as unsigned integers; the two branches together give an exact
// floating-point min.  The branch is taken on the sign bit, not on v >= 0:
// -0.0 compares equal to 0 but its signed-integer image is the most negative
// integer, which would win a signed minimum against every negative value
// already stored.
__device__ __forceinline__ void atomic_min_fp(float* addr, float v) {
    if (!(__float_as_uint(v) >> 31)) atomicMin(reinterpret_cast<int*>(addr), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_min_fp(double* addr, double v) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
    if (!(u >> 63))
        atomicMin(reinterpret_cast<long long*>(addr), __double_as_longlong(v));
    else
        atomicMax(reinterpret_cast<unsigned long long*>(addr), u);
}

// 3-input minimum: one instruction for two candidates in FP32 (PTX min with
// three operands, sm_100 and later); FP64 uses two two-input minima.
__device__ __forceinline__ float min3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(a, fmin(b, c)); }

// Ground cost rho(x,y)^p of an integer offset (dr, dc) >= 0, bracketed:
// lo <= true value <= hi.  p = 1 and p = 2 use correctly rounded operations;
// other p use the FP64 pow (error at most 2 ulp) widened by 2^-49 relative.
template <typename T> struct CostPair { T lo, hi; };

// Brackets of |delta|^p from the exact squared length d2 (an integer below 2^24).
__device__ __forceinline__ CostPair<double> ground_cost_sq_f64(double d2, double p) {
    if (p == 2.0) return {d2, d2};
    if (p == 1.0) return {__dsqrt_rd(d2), __dsqrt_ru(d2)};
    if (d2 == 0.0) return {0.0, 0.0};
    const double c = pow(d2, 0.5 * p);
    return {__dmul_rd(c, 1.0 - 0x1p-49), __dmul_ru(c, 1.0 + 0x1p-49)};
}
__device__ __forceinline__ CostPair<float> ground_cost_sq_f32(double d2, double p) {
    if (p == 2.0) return {(float)d2, (float)d2};            // exact below 2^24
    if (p == 1.0) return {__fsqrt_rd((float)d2), __fsqrt_ru((float)d2)};
    const CostPair<double> c = ground_cost_sq_f64(d2, p);
    return {__double2float_rd(c.lo), __double2float_ru(c.hi)};
}
__device__ __forceinline__ CostPair<double> ground_cost_f64(int dr, int dc, double p) {
    return ground_cost_sq_f64((double)dr * dr + (double)dc * dc, p);   // exact integer
}
__device__ __forceinline__ CostPair<float> ground_cost_f32(int dr, int dc, double p) {
    return ground_cost_sq_f32((double)dr * dr + (double)dc * dc, p);
}

}  // namespace qwb
