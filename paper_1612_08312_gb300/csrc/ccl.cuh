// ccl.cuh -- connected-component labelling helpers shared by the Ising and
// n-vector sweeps.
//
// Labels are union-find parent pointers.  Linking always hangs the larger
// root under the smaller one (atomicMin on the larger root's parent), so the
// root of a finished cluster is its minimum index -- the canonical label.
// Two levels:
//   * tile-local, in shared memory, over tile-local site indices (the local
//     index order agrees with the global one inside a tile);
//   * global, in HBM, over global site indices, for the bonds that cross a
//     tile face.
// Every loop is bounded by UF_MAX_ITERS; exceeding it sets a status bit
// instead of spinning forever.
#pragma once

#include "pyro_internal.cuh"

namespace pyro {

__device__ __forceinline__ int sfind(volatile int *lab, int x)
{
    int p = lab[x];
#pragma unroll 1
    for (int it = 0; p != x && it < UF_MAX_ITERS; ++it) {
        const int gp = lab[p];
        if (gp != p) lab[x] = gp;  // path halving; gp is an ancestor of x
        x = p;
        p = gp;
    }
    return x;
}

// Union of the clusters of a and b in shared memory.  Returns false if the
// iteration bound was hit.
__device__ __forceinline__ bool sunite(int *lab, int a, int b)
{
    volatile int *vl = lab;
#pragma unroll 1
    for (int it = 0; it < 4096; ++it) {
        a = sfind(vl, a);
        b = sfind(vl, b);
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&lab[b], a);
        if (old == b) return true;
        b = old;  // b had been linked meanwhile: unite a with its new parent
    }
    return false;
}

// Global find through L2 (parents can be lowered by other SMs' atomics).
__device__ __forceinline__ int gfind(const int *P, int x)
{
    int p = __ldcg(P + x);
#pragma unroll 1
    for (int it = 0; p != x && it < UF_MAX_ITERS; ++it) {
        x = p;
        p = __ldcg(P + x);
    }
    return x;
}

__device__ __forceinline__ bool gunite(int *P, int a, int b)
{
#pragma unroll 1
    for (int it = 0; it < 65536; ++it) {
        a = gfind(P, a);
        b = gfind(P, b);
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(P + b, a);
        if (old == b) return true;
        b = old;
    }
    return false;
}

// Root of x once no union is in flight (plain cached loads).
__device__ __forceinline__ int root_of(const int *P, int x)
{
    int p = P[x];
#pragma unroll 1
    for (int it = 0; p != x && it < UF_MAX_ITERS; ++it) {
        x = p;
        p = P[x];
    }
    return x;
}

// Warp + block sum of a 64-bit counter into one of NSLOT global slots
// (slots spread the atomics over many addresses).
constexpr int NSLOT = 256;

__device__ __forceinline__ void block_add_u64(unsigned long long v, unsigned long long *slots)
{
    __shared__ unsigned long long red_u64[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) red_u64[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? red_u64[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(slots + (blockIdx.x & (NSLOT - 1)), v);
    }
}

// Deterministic block sum of a double (fixed shuffle tree), result valid in
// thread 0.  Every thread of the block must call it.
__device__ __forceinline__ double block_sum_f64(double v)
{
    __shared__ double red_f64[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red_f64[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? red_f64[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = __dadd_rn(r, __shfl_xor_sync(0xffffffffu, r, o));
    }
    return r;
}

// Neumaier step with explicitly rounded operations (no contraction).
__device__ __forceinline__ void nsum_add(double &s, double &c, double x)
{
    const double t = __dadd_rn(s, x);
    if (fabs(s) >= fabs(x)) c = __dadd_rn(c, __dadd_rn(__dadd_rn(s, -t), x));
    else c = __dadd_rn(c, __dadd_rn(__dadd_rn(x, -t), s));
    s = t;
}

}  // namespace pyro
