// ccl.cuh -- connected-component labelling helpers shared by the Ising and
// n-vector sweeps.
//
// Labels are union-find parent pointers.  Linking always hangs the larger
// root under the smaller one (atomicMin on the larger root's parent), so the
// root of a finished cluster is its minimum index -- the canonical label.
// Two levels:
//   * tile-local, in shared memory, over tile-local site indices (inside a
//     tile the local index order agrees with the global one);
//   * global, in HBM, over global site indices of the tile-local roots of
//     clusters that cross a tile face.
// Every loop is bounded; exceeding a bound sets a status bit instead of
// spinning forever.
#pragma once

#include "pyro_internal.cuh"

namespace pyro {

// Shared-memory slot of tile-local site v = 16 t + s: site-major across the
// tile's cells, so that the 32 threads of a warp (consecutive cells t)
// touch 32 consecutive words for any fixed s (no bank conflicts).
__device__ __forceinline__ int lslot(int v, int nt) { return (v & 15) * nt + (v >> 4); }

__device__ __forceinline__ int sfind(volatile int *lab, int x, int nt)
{
    int p = lab[lslot(x, nt)];
#pragma unroll 1
    for (int it = 0; p != x && it < 65536; ++it) {
        const int gp = lab[lslot(p, nt)];
        if (gp != p) lab[lslot(x, nt)] = gp;  // path halving; gp is an ancestor of x
        x = p;
        p = gp;
    }
    return x;
}

// Union of the clusters of a and b in shared memory.  Returns false if the
// iteration bound was hit.
__device__ __forceinline__ bool sunite(int *lab, int a, int b, int nt)
{
    volatile int *vl = lab;
#pragma unroll 1
    for (int it = 0; it < 4096; ++it) {
        a = sfind(vl, a, nt);
        b = sfind(vl, b, nt);
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&lab[lslot(b, nt)], a);
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
    for (int it = 0; p != x && it < (1 << 20); ++it) {
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

// Root of x once no union is in flight.
__device__ __forceinline__ int root_of(const int *P, int x)
{
    int p = P[x];
#pragma unroll 1
    for (int it = 0; p != x && it < (1 << 20); ++it) {
        x = p;
        p = P[x];
    }
    return x;
}

// Components of a tetrahedron's four vertices under its six bond bits
// (k = 0..5 pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)): rr[v] = smallest
// vertex connected to v.
__device__ __forceinline__ void tet_components(uint32_t bits, int rr[4])
{
    rr[0] = 0;
    rr[1] = 1;
    rr[2] = 2;
    rr[3] = 3;
#pragma unroll
    for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if ((bits >> k) & 1u) {
                const int m = min(rr[pair_a(k)], rr[pair_b(k)]);
                rr[pair_a(k)] = m;
                rr[pair_b(k)] = m;
            }
}

// Pair index k of vertices (a, b), a < b.
__device__ __forceinline__ int pair_index(int a, int b) { return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5); }

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
