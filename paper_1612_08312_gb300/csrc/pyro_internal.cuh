// pyro_internal.cuh -- shared device helpers of libpyro (CUDA, sm_103a).
//
// Lattice index arithmetic (closed form), Philox4x32-10, tile geometry and
// the context structures.  The conventions are those documented in
// include/pyro.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "pyro.h"

namespace pyro {

// Tags of the Philox counter's fourth word.
constexpr uint32_t TAG_BOND = 1u;
constexpr uint32_t TAG_FLIP = 2u;
constexpr uint32_t TAG_AXIS = 3u;
constexpr uint32_t TAG_INIT = 4u;
constexpr uint32_t TAG_TIE = 5u;
constexpr uint32_t INIT_SWEEP_FIELD = 0xFFFFFFFFu;
constexpr int MAX_AXIS_ATTEMPTS = 256;

// Device status bits (see the PYRO_E_* codes).
constexpr int ST_NOCONVERGE = 1;
constexpr int ST_TIMEOUT = 2;

// Bound on union-find loop iterations; every real case needs a few dozen.
constexpr int UF_MAX_ITERS = 1 << 22;

// ---------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// two-multiplier S-box on a 4x32-bit counter, key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hiA = __umulhi(0xD2511F53u, c.x);
        const uint32_t loA = 0xD2511F53u * c.x;
        const uint32_t hiB = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t loB = 0xCD9E8D57u * c.z;
        c = make_uint4(hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA);
    }
    return c;
}

// Call j of the stream (seed, sweep field, tag).
__device__ __forceinline__ uint4 philox_call(uint64_t seed, uint32_t sweep, uint32_t tag, uint64_t j)
{
    return philox(make_uint4((uint32_t)j, (uint32_t)(j >> 32), sweep, tag), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(uint4 w, int slot)
{
    return slot == 0 ? w.x : slot == 1 ? w.y : slot == 2 ? w.z : w.w;
}

// ------------------------------------------------------------- geometry --
// FCC sub-point f of a cubic cell sits at A_f = 2 a(f) (quarter-cell units)
// with a(1) = (0,1,1), a(2) = (1,0,1), a(3) = (1,1,0); a is linear over
// GF(2) in the bits of f, so A_f - A_nu = A_{f^nu} - 4 h with h in {0,1}^3.
__host__ __device__ constexpr int afcc(int f, int d)
{
    return d == 0 ? ((f >> 1) & 1) : d == 1 ? (f & 1) : (((f & 1) ^ (f >> 1)) & 1);
}

// The tetrahedron through site (cell c, f, basis 0) other than its own
// "up" one has vertex nu (nu = 1..3) at cell c - h(f, nu), FCC sub-point
// f ^ nu, basis nu; h_d = 1 iff a_d(f) = 0 and a_d(nu) = 1.  Returned as a
// 3-bit mask (bit d = backward step along axis d).
__host__ __device__ constexpr int down_shift_mask(int f, int nu)
{
    return ((afcc(f, 0) == 0 && afcc(nu, 0) == 1) ? 1 : 0) |
           ((afcc(f, 1) == 0 && afcc(nu, 1) == 1) ? 2 : 0) |
           ((afcc(f, 2) == 0 && afcc(nu, 2) == 1) ? 4 : 0);
}

// Bit (site offset in its cell) of vertex v of the down tetrahedron of f.
__host__ __device__ constexpr int down_bit(int f, int v) { return v == 0 ? 4 * f : 4 * (f ^ v) + v; }
// Cell shift mask of vertex v of the down tetrahedron of f.
__host__ __device__ constexpr int down_mask(int f, int v) { return v == 0 ? 0 : down_shift_mask(f, v); }

// Vertex pairs of the six bonds of a tetrahedron, k = 0..5.
__host__ __device__ constexpr int pair_a(int k) { return k < 3 ? 0 : (k < 5 ? 1 : 2); }
__host__ __device__ constexpr int pair_b(int k) { return k < 3 ? k + 1 : (k < 5 ? k - 1 : 3); }

// ------------------------------------------------------------- contexts --
struct DevStats {
    unsigned long long sweep;  // sweep field of the next sweep's Philox counters
    unsigned long long epoch;       // stamp of the next sweep's crossing-cluster links
    unsigned long long last_epoch;  // stamp of the last completed sweep's links
    int status;                // ST_* bits
    int pad;
    // accumulators (Neumaier): E, E^2, m^2, m^4, |m|
    double acc_s[5];
    double acc_c[5];
    unsigned long long count;
    // last measurement: E, m2, m4, M_x
    double last[4];
};

struct TileShape {
    int TX, TY, TZ;
};

// One lattice (replica) as the kernels see it.
struct Rep {
    void *spins;       // Ising: uint16 per cell; n-vector: n planes of N values
    uint16_t *L16;     // per site: tile-local index of its tile-local root (13 bits);
                       // on a root whose cluster crosses a tile face, bit 14 =
                       // the cluster's flip bit XOR the root's own flip bit
    unsigned long long *P;  // crossing-cluster links: (epoch stamp << 32) | parent
    uint16_t *F;       // the sweep's flip bit of every site, one word per cell
    uint32_t *dmask;   // union pairs of face cells that cross the tile (24 bits)
    int32_t *labels;   // canonical labels (filled on demand), or NULL
    DevStats *st;
    double *trace;     // ring buffer of (E, m2, m4, M_x), or NULL
    int64_t trace_cap;
    uint64_t seed;
    uint64_t thr;      // Ising bond threshold floor((1 - exp(-2 beta J)) 2^32), <= 2^32
    double K2;         // 2 beta J
    double J;
    int64_t N, ncells;
    int L, ntx, nty, pad;
};

// Up to MAX_REPS lattices updated by one launch per phase.  Blocks of the
// tiled kernels map to (replica, tile) through tile_begin; blocks of the
// per-cell kernels (256 cells each) through block_begin.  Tile edges are
// powers of two that divide every replica's L.
constexpr int MAX_REPS = 64;
constexpr int CELL_BLOCK = 256;

struct Batch {
    const Rep *reps;
    double *partials;  // 4 per tile
    int R, TX, TY, TZ;
    int lTX, lTY, lTZ;  // log2 of the (power-of-two) tile edges
    int64_t tile_begin[MAX_REPS + 1];
    int64_t block_begin[MAX_REPS + 1];
    // last, so that the fields the sweep kernels read keep their offsets
    // (moving them measurably slowed the local and crossing kernels)
    double *folded;    // 4 per group of a replica's partials (fold groups per replica), or unused
    int fold;          // groups per replica the partials are first summed into; 0 = none
};

__device__ __forceinline__ int find_rep(const int64_t *begin, int R, int64_t blk)
{
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace pyro

namespace pyro {

// Thread-local last-error message.
void set_error(const std::string &msg);

// Largest dynamic shared memory a block may opt into on the current device.
// Kernels' MaxDynamicSharedMemorySize attributes are set to this value (a
// per-function setting that must never be lowered below what another
// lattice's tile needs).
inline int smem_optin()
{
    int dev = 0, v = 48 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Let kernel k take up to `need` bytes of dynamic shared memory: invalid if
// that and its static shared memory exceed the opt-in limit, else the
// attribute is raised to what the static part leaves.
template <typename K>
inline cudaError_t allow_dynamic_smem(K k, size_t need)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    const int room = smem_optin() - (int)a.sharedSizeBytes;
    if ((int)need > room) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

}  // namespace pyro
