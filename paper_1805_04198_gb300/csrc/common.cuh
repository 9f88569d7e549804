// common.cuh -- numerics and small helpers shared by the libeik kernels.
//
// The local solver below is the Godunov upwind solve of Sec. 1.1 (eq.
// "godonuv") in the closed form of Sec. 3.2 (definition of C_H) with the
// per-axis neighbour choice of Alg. 3.  Every multiply and add is written with
// an explicitly rounded intrinsic so the compiler can never contract a pair
// into a fused multiply-add: the FP64 build then performs exactly the IEEE
// operations the method is defined by, in the order written here.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eik {

constexpr unsigned FULL = 0xffffffffu;

template <class T> struct Num;

template <> struct Num<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

template <> struct Num<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

// Wind packing: component a in {-1,0,+1} stored as (w+1) in 2 bits at 2a.
// Sign = direction of travel: +1 when the upwind (smaller) neighbour is on the
// minus side of the axis.
__host__ __device__ __forceinline__ uint8_t wind_pack(int wx, int wy, int wz = 0) {
    return (uint8_t)((wx + 1) | ((wy + 1) << 2) | ((wz + 1) << 4));
}
__host__ __device__ __forceinline__ int wind_comp(uint8_t w, int a) { return (int)((w >> (2 * a)) & 3) - 1; }
constexpr uint8_t WIND_ZERO = 0x15;  // (0,0,0)

// 2-D Godunov local solve.  vm*/vp* are the neighbours on the minus/plus side
// of each axis (+inf where missing: the one-sided rule of Sec. 1.1).  Returns
// u~ and the packed wind of the branch taken (zero wind when u~ is +inf).
template <class T>
__device__ __forceinline__ T local_solve2(T vmx, T vpx, T vmy, T vpy, T rh, uint8_t &wind) {
    using N = Num<T>;
    T a, b;
    int sa, sb;
    // Alg. 3: the smaller neighbour per axis; a tie goes to the plus side.
    if (vmx < vpx) { a = vmx; sa = 1; } else { a = vpx; sa = -1; }
    if (vmy < vpy) { b = vmy; sb = 1; } else { b = vpy; sb = -1; }
    T d = N::sub(a, b);
    T u;
    if (fabs(d) < rh) {
        // two-term branch: (a + b + sqrt(2 r^2 h^2 - (a-b)^2)) / 2
        T disc = N::sub(N::mul(N::mul(T(2), rh), rh), N::mul(d, d));
        u = N::mul(N::add(N::add(a, b), N::sqrt_(disc)), T(0.5));
        wind = wind_pack(sa, sb);
    } else if (a < b) {
        u = N::add(a, rh);
        wind = (u < N::inf()) ? wind_pack(sa, 0) : WIND_ZERO;
    } else {
        u = N::add(b, rh);
        wind = (u < N::inf()) ? wind_pack(0, sb) : WIND_ZERO;
    }
    return u;
}

// Value-only variant used inside the sweeps (the wind is recomputed from the
// converged state, so the sweeps need only the value).
template <class T>
__device__ __forceinline__ T local_solve2_value(T vmx, T vpx, T vmy, T vpy, T rh) {
    using N = Num<T>;
    T a = fmin(vmx, vpx);
    T b = fmin(vmy, vpy);
    T d = N::sub(a, b);
    if (fabs(d) < rh) {
        T disc = N::sub(N::mul(N::mul(T(2), rh), rh), N::mul(d, d));
        return N::mul(N::add(N::add(a, b), N::sqrt_(disc)), T(0.5));
    }
    return N::add(fmin(a, b), rh);
}

// Status codes mirrored from eik.h for device code.
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = -4;

// Bounded spin limit for every device-side wait (iterations of ~64 ns sleep).
constexpr long long SPIN_LIMIT = 1ll << 22;

}  // namespace eik
