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
    // Square root used inside the local solve.  FP32 storage carries a 1e-5
    // accuracy budget, so the single-instruction hardware approximation
    // (relative error ~1e-7, applied only to the increment of the two-term
    // branch) is used; FP64 keeps the correctly rounded root.
    static __device__ __forceinline__ float sqrt_solve(float a) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
};

template <> struct Num<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ double sqrt_solve(double a) { return __dsqrt_rn(a); }
};

// Wind packing: component a in {-1,0,+1} stored as (w+1) in 2 bits at 2a.
// Sign = direction of travel: +1 when the upwind (smaller) neighbour is on the
// minus side of the axis.
__host__ __device__ __forceinline__ uint8_t wind_pack(int wx, int wy, int wz = 0) {
    return (uint8_t)((wx + 1) | ((wy + 1) << 2) | ((wz + 1) << 4));
}
__host__ __device__ __forceinline__ int wind_comp(uint8_t w, int a) { return (int)((w >> (2 * a)) & 3) - 1; }
constexpr uint8_t WIND_ZERO = 0x15;  // (0,0,0)
// Flag on a subdomain's copy of a coarse-set node (never on W or w^k): the node
// was inflow and the subdomain solve kept its Step 2 value U, so the copy
// echoes boundary data rather than a fine solution.
constexpr uint8_t WIND_ECHO = 0x80;

// 2-D Godunov local solve.  vm*/vp* are the neighbours on the minus/plus side
// of each axis (+inf where missing: the one-sided rule of Sec. 1.1).  Returns
// u~ and the packed wind of the branch taken (zero wind when u~ is +inf).
// Both branches are evaluated and one is selected, so no warp diverges; the
// selected branch performs exactly the operations written in the paper's
// closed form.
template <class T>
__device__ __forceinline__ T local_solve2(T vmx, T vpx, T vmy, T vpy, T rh, uint8_t &wind) {
    using N = Num<T>;
    // Alg. 3: the smaller neighbour per axis; a tie goes to the plus side.
    const bool lx = vmx < vpx, ly = vmy < vpy;
    const T a = lx ? vmx : vpx, b = ly ? vmy : vpy;
    const int sa = lx ? 1 : -1, sb = ly ? 1 : -1;
    const T d = N::sub(a, b);
    // two-term branch: (a + b + sqrt(2 r^2 h^2 - (a-b)^2)) / 2
    const T disc = N::sub(N::mul(N::mul(T(2), rh), rh), N::mul(d, d));
    const T u2 = N::mul(N::add(N::add(a, b), N::sqrt_solve(fmax(disc, T(0)))), T(0.5));
    const bool two = fabs(d) < rh;
    const bool ax = a < b;
    const T u1 = N::add(ax ? a : b, rh);
    const T u = two ? u2 : u1;
    wind = two ? wind_pack(sa, sb) : (u < N::inf() ? (ax ? wind_pack(sa, 0) : wind_pack(0, sb)) : WIND_ZERO);
    return u;
}

// Value-only variant used inside the sweeps (the wind is recomputed from the
// converged state, so the sweeps need only the value).
template <class T>
__device__ __forceinline__ T local_solve2_value(T vmx, T vpx, T vmy, T vpy, T rh) {
    using N = Num<T>;
    const T a = fmin(vmx, vpx);
    const T b = fmin(vmy, vpy);
    const T d = N::sub(a, b);
    const T disc = N::sub(N::mul(N::mul(T(2), rh), rh), N::mul(d, d));
    const T u2 = N::mul(N::add(N::add(a, b), N::sqrt_solve(fmax(disc, T(0)))), T(0.5));
    const T u1 = N::add(fmin(a, b), rh);
    return fabs(d) < rh ? u2 : u1;
}

// 3-D Godunov local solve: axis minima sorted a_p0 <= a_p1 <= a_p2 (ties keep
// axis order); one term, else the paper's two-term formula on the two
// smallest, else the three-term quadratic written in t = u - a_p0:
//   t^2 + (t - d1)^2 + (t - d2)^2 = (r h)^2.
// The wind has the per-axis sign of Alg. 3 on the axes used.  With a_p2 = inf
// it reduces exactly to local_solve2.  The sort is done by ranks and selects
// (no indexed local arrays); the arithmetic is the same sequence of rounded
// operations on the sorted values.
template <class T>
__device__ __forceinline__ T local_solve3(const T *vm, const T *vp, T rh, uint8_t &wind) {
    using N = Num<T>;
    const bool l0 = vm[0] < vp[0], l1 = vm[1] < vp[1], l2 = vm[2] < vp[2];
    const T a0 = l0 ? vm[0] : vp[0], a1 = l1 ? vm[1] : vp[1], a2 = l2 ? vm[2] : vp[2];
    // stable ranks: axis b precedes axis c when a_b < a_c, or a_b == a_c and b < c
    const int r0 = (a1 < a0 ? 1 : 0) + (a2 < a0 ? 1 : 0);
    const int r1 = (a0 <= a1 ? 1 : 0) + (a2 < a1 ? 1 : 0);
    const int r2 = (a0 <= a2 ? 1 : 0) + (a1 <= a2 ? 1 : 0);
    const T v0 = r0 == 0 ? a0 : (r1 == 0 ? a1 : a2);
    const T v1 = r0 == 1 ? a0 : (r1 == 1 ? a1 : a2);
    const T v2 = r0 == 2 ? a0 : (r1 == 2 ? a1 : a2);
    const T d01 = N::sub(v0, v1);
    const bool two = fabs(d01) < rh;
    const T disc = N::sub(N::mul(N::mul(T(2), rh), rh), N::mul(d01, d01));
    const T u2 = N::mul(N::add(N::add(v0, v1), N::sqrt_solve(fmax(disc, T(0)))), T(0.5));
    const T u1 = N::add(v0, rh);
    const bool three = two && (u2 > v2);
    T u = two ? u2 : u1;
    if (three) {
        const T d1 = N::sub(v1, v0);
        const T d2 = N::sub(v2, v0);
        const T sd = N::add(d1, d2);
        T disc3 = N::sub(N::mul(sd, sd), N::mul(T(3), N::sub(N::add(N::mul(d1, d1), N::mul(d2, d2)), N::mul(rh, rh))));
        if (disc3 < T(0)) disc3 = T(0);
        u = N::add(v0, N::div(N::add(sd, N::sqrt_solve(disc3)), T(3)));
    }
    const int nt = three ? 3 : (two ? 2 : (u < N::inf() ? 1 : 0));  // axes used, by rank
    wind = wind_pack(r0 < nt ? (l0 ? 1 : -1) : 0, r1 < nt ? (l1 ? 1 : -1) : 0, r2 < nt ? (l2 ? 1 : -1) : 0);
    return u;
}

// Register cap of a sweep-engine kernel by element type (FP32, FP64): keeps
// the single-CTA launch shapes (up to 32 warps) and the co-residency of the
// cooperative multi-CTA forms.
template <class T, int F32, int F64> struct RegCap {
    static constexpr int v = sizeof(T) == 4 ? F32 : F64;
};

// Status codes mirrored from eik.h for device code.
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = -4;

// Default iteration limit of every bounded device-side wait (iterations of at
// most ~1 us sleep each, so an expired wait reports within seconds).
constexpr long long SPIN_LIMIT_DEFAULT = 1ll << 22;

// The limit in force.  Each translation unit that waits has its own copy per
// device; eik_set_wait_limit writes every copy through the setter that the
// unit defines with EIK_SPIN_LIMIT_SETTER.  A kernel that waits reads it once
// when it starts (a global load on the path of a wait would delay the wait
// itself).
static __device__ long long g_spin_limit = SPIN_LIMIT_DEFAULT;
__device__ __forceinline__ long long spin_limit() { return *(volatile const long long *)&g_spin_limit; }
#define EIK_SPIN_LIMIT_SETTER(fname) \
    int fname(long long v) { return (int)cudaMemcpyToSymbol(g_spin_limit, &v, sizeof(v)); }

// Grid-wide barrier for cooperative launches (all CTAs co-resident).  bar[0]
// counts arrivals, bar[1] is the generation.  The wait is bounded by `lim`
// polls (the kernel reads spin_limit() once when it starts): on timeout the
// error word is set and false is returned to every thread of the CTA (the
// caller then returns with the whole CTA).
__device__ inline bool grid_barrier(unsigned *bar, int *err, long long lim) {
    __shared__ int s_barrier_ok;
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*vgen == gen) {
                if (++it > lim) {
                    atomicExch(err, DEV_TIMEOUT);
                    ok = false;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_barrier_ok = ok ? 1 : 0;
    }
    __syncthreads();
    ok = s_barrier_ok != 0;
    __syncthreads();  // s_barrier_ok is read by all before the next barrier writes it
    return ok;
}

// Per-node weight of Sec. 4.2 from du = u^k - u^{k-1} and the last n changes
// dC[s] of C_H(nbrs U): eq. secthetaest (weighted mean of the changes), the
// damping of eq. thetaest, the optional cap; `fallback` where undefined.  A is
// any argument block carrying the weights om[3] and the damping parameters sg
// (gamma), sd (delta), sx0 (x0) and cap.
template <class Args>
__device__ inline double theta_estimate(const Args &A, double du, const double *dC, int n, double fallback) {
    double den = 0.0, wsum = 0.0;
    for (int s = 0; s < n; ++s) {
        den = __dadd_rn(den, __dmul_rn(A.om[s], dC[s]));
        wsum = __dadd_rn(wsum, A.om[s]);
    }
    if (!(wsum > 0.0)) return fallback;
    den = __ddiv_rn(den, wsum);
    const double t = __ddiv_rn(du, den);
    if (!isfinite(t) || den == 0.0) return fallback;
    const double sig = __ddiv_rn(1.0, __dadd_rn(1.0, exp(__ddiv_rn(__dsub_rn(t, A.sx0), A.sg))));
    double v = __dadd_rn(__dmul_rn(sig, t), __dmul_rn(__dmul_rn(__dsub_rn(1.0, sig), A.sd), t));
    if (A.cap > 0.0 && v > A.cap) v = A.cap;
    return v > 0.0 ? v : 0.0;
}

}  // namespace eik
