// nvec.cuh -- n-vector arithmetic shared by the pyrochlore and the
// generic-lattice sweeps (Eq. 1 with n = 2, 3; Wolff's embedded cluster):
// explicitly rounded FP64 operations (no fused multiply-add, so results are
// those of a plain IEEE evaluation in the written order) or plain FP32, the
// per-sweep random axis, projections and bond thresholds.
#pragma once

#include "pyro_internal.cuh"

namespace pyro {

template <typename T>
struct Ar;

template <>
struct Ar<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dadd_rn(a, -b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double bond_p(double K2, double x) { return -expm1(-__dmul_rn(K2, x)); }
};

template <>
struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float div(float a, float b) { return a / b; }
    static __device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
    static __device__ __forceinline__ float bond_p(float K2, float x) { return -expm1f(-(K2 * x)); }
};

// Uniform unit vector from the (seed, sweep, tag) stream, FP64 with
// correctly rounded operations: rejection in the square, then n = 2:
// (u0, u1)/sqrt(s); n = 3: Marsaglia's (2 u0 sqrt(1-s), 2 u1 sqrt(1-s), 1-2s).
template <int NC>
__device__ __forceinline__ void unit_vector_dev(uint64_t seed, uint32_t sweep, uint32_t tag, uint64_t call_base,
                                                double r[3])
{
#pragma unroll 1
    for (int att = 0; att < MAX_AXIS_ATTEMPTS; ++att) {
        const uint4 w = philox_call(seed, sweep, tag, call_base + (uint64_t)att);
        const double u0 = (double)(int32_t)w.x * 4.656612873077392578125e-10;
        const double u1 = (double)(int32_t)w.y * 4.656612873077392578125e-10;
        const double s = __dadd_rn(__dmul_rn(u0, u0), __dmul_rn(u1, u1));
        if (s > 0.0 && s < 1.0) {
            if (NC == 2) {
                const double q = __dsqrt_rn(s);
                r[0] = __ddiv_rn(u0, q);
                r[1] = __ddiv_rn(u1, q);
                r[2] = 0.0;
            } else {
                const double t = __dsqrt_rn(__dadd_rn(1.0, -s));
                r[0] = __dmul_rn(__dmul_rn(2.0, u0), t);
                r[1] = __dmul_rn(__dmul_rn(2.0, u1), t);
                r[2] = __dadd_rn(1.0, -__dmul_rn(2.0, s));
            }
            return;
        }
    }
    r[0] = 1.0;
    r[1] = 0.0;
    r[2] = 0.0;
}

template <int NC, typename T>
__device__ __forceinline__ T project(const T *spins, int64_t N, int64_t i, const T r[3])
{
    using A = Ar<T>;
    T p = A::mul(spins[i], r[0]);
#pragma unroll
    for (int k = 1; k < NC; ++k) p = A::add(p, A::mul(spins[k * N + i], r[k]));
    return p;
}

// Threshold of a bond with activation probability p: active iff its 32-bit
// uniform w < floor(p 2^32) (p = 1 gives 2^32).
__device__ __forceinline__ uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    const double t = floor(__dmul_rn(p, 4294967296.0));
    return t >= 4294967296.0 ? (1ull << 32) : (uint64_t)t;
}

__device__ __forceinline__ uint64_t prob_threshold(float p)
{
    if (!(p > 0.0f)) return 0;
    if (p >= 1.0f) return 1ull << 32;
    // p < 1: p 2^32 (exact, a power-of-two scaling) is below 2^32, and the
    // truncating conversion is the floor
    return __float2uint_rz(p * 4294967296.0f);
}

}  // namespace pyro
