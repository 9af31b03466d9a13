// ccl.cuh -- connected-component labelling helpers shared by the Ising and
// n-vector sweeps.
//
// Labels are union-find parent pointers.  Linking always hangs the larger
// root under the smaller one (atomicMin on the larger root's parent), so the
// root of a finished cluster is its minimum index -- the canonical label.
// This file holds the tile-local level, in shared memory, over tile-local
// site indices (inside a tile the local index order agrees with the global
// one); the global level for clusters that cross tile faces is in
// sweep_core.cuh.  Every loop is bounded; exceeding a bound sets a status
// bit instead of spinning forever.
#pragma once

#include "pyro_internal.cuh"

namespace pyro {

// Shared-memory slot of tile-local site v = 16 t + s: site-major across the
// tile's cells, so that the 32 threads of a warp (consecutive cells t)
// touch 32 consecutive words for any fixed s (no bank conflicts).
__device__ __forceinline__ int lslot(int v, int nt) { return (v & 15) * nt + (v >> 4); }

// Iteration bound of one union (4096).  A test can lower it (to 0) through
// pyro_debug_set to exercise the bound-exceeded status path.
static __constant__ int c_unite_bound = 4096;

// Union of the clusters of a and b in shared memory.  Both finds walk in
// lockstep, so their shared-memory loads overlap; they write nothing on the
// way (path-halving writes were measured slower: the final resolution of
// the representatives shortens the trees once, for all of them).
// Returns false if the iteration bound was hit.
__device__ __forceinline__ bool sunite(int *lab, int a, int b, int nt)
{
    volatile int *vl = lab;
    const int bound = c_unite_bound;
    int pa = vl[lslot(a, nt)], pb = vl[lslot(b, nt)];
#pragma unroll 1
    for (int it = 0; it < bound; ++it) {
#pragma unroll 1
        for (int st = 0; (pa != a || pb != b) && st < 65536; ++st) {
            if (pa != a) {
                const int g = vl[lslot(pa, nt)];
                a = pa;
                pa = g;
            }
            if (pb != b) {
                const int g = vl[lslot(pb, nt)];
                b = pb;
                pb = g;
            }
        }
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&lab[lslot(b, nt)], a);
        if (old == b) return true;
        // b had been linked meanwhile: unite a with its new parent
        b = old;
        pa = vl[lslot(a, nt)];
        pb = vl[lslot(b, nt)];
    }
    return false;
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
