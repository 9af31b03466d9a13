// vector.cu -- Swendsen-Wang sweep of the pyrochlore XY (n = 2) and
// Heisenberg (n = 3) models with Wolff's embedded-cluster construction
// (Sec. 2): per sweep one random unit axis r; the projections p_i = s_i.r
// define an Ising model with couplings J p_i p_j; bonds with p_i p_j > 0 are
// activated with probability 1 - exp(-2 beta J p_i p_j); flipped clusters
// reflect their spins, s -> s - 2 (s.r) r.
//
// Spins are stored as n component planes of N values of T (float or
// double).  A bond with p_i p_j > 0 is active iff its 32-bit uniform
// w < floor(p 2^32), w drawn like the Ising bonds' (sweep_core.cuh).  The FP64 path uses explicitly rounded IEEE operations in the
// same order as the definition, so projections, reflections and the axis
// are bit-identical to a straightforward FP64 evaluation without fused
// multiply-add.  The FP32 path stores and updates spins in float; its
// measurements are accumulated in FP64.
//
// Kernels (each over a Batch of lattices): vec_local (projections of the
// tile + halo staged in shared memory, bond activation, tile-local
// labelling), the global union of tile-crossing clusters (boundary_kernel,
// shared with the Ising sweep), vec_flip (root, flip, reflection) and
// vec_measure (E and M per block in FP64).
#include "sweep_core.cuh"

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
    const float t = floorf(p * 4294967296.0f);
    return t >= 4294967296.0f ? (1ull << 32) : (uint64_t)__float2ull_rz(t);
}

template <typename T>
__host__ __device__ constexpr size_t vec_halo_bytes(int TX, int TY, int TZ)
{
    return (size_t)16 * (TX + 1) * (TY + 1) * (TZ + 1) * sizeof(T);
}

template <int NC, typename T>
__global__ void __launch_bounds__(512) vec_local_kernel(const __grid_constant__ Batch B)
{
    using A = Ar<T>;
    extern __shared__ __align__(16) int smem[];
    const int rep = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[rep]);
    const int nt = c.nt, L = c.L;
    const int64_t N = R.N;
    int *lab = smem;
    uint32_t *plist = reinterpret_cast<uint32_t *>(smem + 16 * nt);
    int *pcount = smem + 28 * nt;
    T *proj = reinterpret_cast<T *>(smem + 28 * nt + 4);
    const int HX = c.TX + 1, HY = c.TY + 1, HZ = c.TZ + 1;
    const T *spins = static_cast<const T *>(R.spins);
    const uint32_t sweep = (uint32_t)R.st->sweep;
    const uint64_t seed = R.seed;

    double rd[3];
    unit_vector_dev<NC>(seed, sweep, TAG_AXIS, 0, rd);
    const T r[3] = {(T)rd[0], (T)rd[1], (T)rd[2]};

    // projections s_i . r of the tile's sites and the backward halo
    for (int idx = threadIdx.x; idx < 16 * HX * HY * HZ; idx += blockDim.x) {
        const int h = idx >> 4, s = idx & 15;
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        int gx = c.ox + hx - 1, gy = c.oy + hy - 1, gz = c.oz + hz - 1;
        gx += (gx < 0) ? L : 0;
        gy += (gy < 0) ? L : 0;
        gz += (gz < 0) ? L : 0;
        const int64_t i = 16 * ((int64_t)gx + (int64_t)L * ((int64_t)gy + (int64_t)L * gz)) + s;
        proj[idx] = project<NC, T>(spins, N, i, r);
    }
    __syncthreads();

    // halo cell of the vertex at backward-shift mask m
    auto hidx = [&](int m) {
        return (c.lx + 1 - (m & 1)) + HX * ((c.ly + 1 - ((m >> 1) & 1)) + HY * (c.lz + 1 - ((m >> 2) & 1)));
    };
    const T K2 = (T)R.K2;
    uint64_t act = 0;
    if (R.K2 > 0.0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            T xq[8];
            uint32_t pos = 0;
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int cb = 8 * q + h, f = cb / 12, k = cb % 12;
                const bool up = k < 6;
                const int kk = up ? k : k - 6;
                const int va = pair_a(kk), vb = pair_b(kk);
                const T pa = up ? proj[16 * hidx(0) + 4 * f + va] : proj[16 * hidx(down_mask(f, va)) + down_bit(f, va)];
                const T pb = up ? proj[16 * hidx(0) + 4 * f + vb] : proj[16 * hidx(down_mask(f, vb)) + down_bit(f, vb)];
                xq[h] = A::mul(pa, pb);
                pos |= (xq[h] > (T)0 ? 1u : 0u) << h;
            }
            if (!pos) continue;
            const uint64_t j = 6 * (uint64_t)c.cell + q;
            const uint4 wd = philox_call(seed, sweep, TAG_BOND, j);
            const uint32_t ww[4] = {wd.x, wd.y, wd.z, wd.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                if (!((pos >> h) & 1u)) continue;
                const HalfCompare hc(prob_threshold(A::bond_p(K2, xq[h])));
                const uint32_t hi = (ww[h >> 1] >> (16 * (h & 1))) & 0xFFFFu;
                bool a = hc.all || hi < hc.thi;
                if (!hc.all && hi == hc.thi) {
                    const uint4 wt = philox_call(seed, sweep, TAG_TIE, j);
                    a = ((word_of(wt, h >> 1) >> (16 * (h & 1))) & 0xFFFFu) < hc.tlo;
                }
                act |= (uint64_t)(a ? 1u : 0u) << (8 * q + h);
            }
        }
    }
    local_core(c, R, act, sweep, lab, plist, pcount);
}

template <int NC, typename T>
__global__ void __launch_bounds__(512) vec_flip_kernel(const __grid_constant__ Batch B)
{
    using A = Ar<T>;
    extern __shared__ __align__(16) int smem[];
    const int rep = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[rep]);
    uint16_t *ls = reinterpret_cast<uint16_t *>(smem);
    uint16_t *fs = ls + 16 * c.nt;
    int root[16];
    uint32_t flip;
    resolve_cell(c, R, ls, fs, root, flip);
    if (!flip) return;
    double rd[3];
    unit_vector_dev<NC>(R.seed, (uint32_t)R.st->sweep, TAG_AXIS, 0, rd);
    const T r[3] = {(T)rd[0], (T)rd[1], (T)rd[2]};
    T *spins = static_cast<T *>(R.spins);
    const int64_t N = R.N;
    while (flip) {
        const int s = __ffs(flip) - 1;
        flip &= flip - 1;
        const int64_t i = 16 * c.cell + s;
        const T pr = project<NC, T>(spins, N, i, r);
        const T d2 = A::mul((T)2, pr);
        T sv[3];
#pragma unroll
        for (int k = 0; k < NC; ++k) sv[k] = A::sub(spins[k * N + i], A::mul(d2, r[k]));
        T q = A::mul(sv[0], sv[0]);
#pragma unroll
        for (int k = 1; k < NC; ++k) q = A::add(q, A::mul(sv[k], sv[k]));
        q = A::sqrt_(q);
#pragma unroll
        for (int k = 0; k < NC; ++k) spins[k * N + i] = A::div(sv[k], q);
    }
}

// Energy (Eq. 1) and magnetisation of the current configuration: every
// cell sums the 48 bonds it owns and its 16 spins in FP64; one partial
// (E, M_x, M_y, M_z) per block.
template <int NC, typename T>
__global__ void __launch_bounds__(CELL_BLOCK) vec_measure_kernel(const __grid_constant__ Batch B)
{
    const int rep = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const int64_t cell = (blockIdx.x - B.block_begin[rep]) * CELL_BLOCK + threadIdx.x;
    double e = 0.0, M[3] = {0.0, 0.0, 0.0};
    if (cell < R.ncells) {
        const int L = R.L;
        const int64_t N = R.N;
        const T *sp = static_cast<const T *>(R.spins);
        const int x = (int)(cell % L), y = (int)((cell / L) % L), z = (int)(cell / ((int64_t)L * L));
        int64_t cb[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int cx = (m & 1) ? (x == 0 ? L - 1 : x - 1) : x;
            const int cy = (m & 2) ? (y == 0 ? L - 1 : y - 1) : y;
            const int cz = (m & 4) ? (z == 0 ? L - 1 : z - 1) : z;
            cb[m] = 16 * ((int64_t)cx + (int64_t)L * ((int64_t)cy + (int64_t)L * cz));
        }
#pragma unroll
        for (int s = 0; s < 16; ++s)
#pragma unroll
            for (int k = 0; k < NC; ++k) M[k] += (double)sp[k * N + 16 * cell + s];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int va = pair_a(k), vb = pair_b(k);
                // up tetrahedron
                const int64_t iu = 16 * cell + 4 * f + va, ju = 16 * cell + 4 * f + vb;
                T du = sp[iu] * sp[ju];
#pragma unroll
                for (int c = 1; c < NC; ++c) du += sp[c * N + iu] * sp[c * N + ju];
                // down tetrahedron
                const int64_t id = cb[down_mask(f, va)] + down_bit(f, va);
                const int64_t jd = cb[down_mask(f, vb)] + down_bit(f, vb);
                T dd = sp[id] * sp[jd];
#pragma unroll
                for (int c = 1; c < NC; ++c) dd += sp[c * N + id] * sp[c * N + jd];
                e += (double)du + (double)dd;
            }
        }
    }
    const double se = block_sum_f64(e);
    const double s0 = block_sum_f64(M[0]);
    const double s1 = block_sum_f64(M[1]);
    const double s2 = block_sum_f64(M[2]);
    if (threadIdx.x == 0) {
        double *o = B.partials + 4 * (int64_t)blockIdx.x;
        o[0] = se;
        o[1] = s0;
        o[2] = s1;
        o[3] = s2;
    }
}

// Ordered start (e_x) or Philox-random start: site i takes attempt a of
// call index (i << 8) | a of the INIT stream.
template <int NC, typename T>
__global__ void __launch_bounds__(CELL_BLOCK) vec_init_kernel(const __grid_constant__ Batch B, int random)
{
    const int rep = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const int64_t cell = (blockIdx.x - B.block_begin[rep]) * CELL_BLOCK + threadIdx.x;
    if (cell >= R.ncells) return;
    T *spins = static_cast<T *>(R.spins);
    for (int s = 0; s < 16; ++s) {
        const int64_t i = 16 * cell + s;
        double r[3] = {1.0, 0.0, 0.0};
        if (random) unit_vector_dev<NC>(R.seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i << 8, r);
#pragma unroll
        for (int k = 0; k < NC; ++k) spins[k * R.N + i] = (T)r[k];
    }
}

// ------------------------------------------------------------ launchers --
size_t resolve_smem(const TileShape &t);
void launch_boundary(int unite, const Batch &B, int64_t ntiles, cudaStream_t s);

size_t vec_local_smem(const TileShape &t, int prec)
{
    const int nt = t.TX * t.TY * t.TZ;
    return core_smem_bytes(nt) +
           (prec == PYRO_FP64 ? vec_halo_bytes<double>(t.TX, t.TY, t.TZ) : vec_halo_bytes<float>(t.TX, t.TY, t.TZ));
}

template <int NC, typename T>
struct VecOps {
    static cudaError_t prepare(const TileShape &t, int prec)
    {
        cudaError_t e = cudaFuncSetAttribute(vec_local_kernel<NC, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)vec_local_smem(t, prec));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(vec_flip_kernel<NC, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)resolve_smem(t));
        return e;
    }
    static void init(const Batch &B, int64_t nblocks, int random, cudaStream_t s)
    {
        vec_init_kernel<NC, T><<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B, random);
    }
    static void phase(int p, const Batch &B, int64_t ntiles, int prec, cudaStream_t s)
    {
        const TileShape t{B.TX, B.TY, B.TZ};
        const int nt = B.TX * B.TY * B.TZ;
        if (p == 0) vec_local_kernel<NC, T><<<(unsigned)ntiles, nt, vec_local_smem(t, prec), s>>>(B);
        else if (p == 1 || p == 2) launch_boundary(p == 2, B, ntiles, s);
        else vec_flip_kernel<NC, T><<<(unsigned)ntiles, nt, resolve_smem(t), s>>>(B);
    }
    static void measure(const Batch &B, int64_t nblocks, cudaStream_t s)
    {
        vec_measure_kernel<NC, T><<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B);
    }
};

#define PYRO_VEC_DISPATCH(model, prec, call)                                       \
    do {                                                                            \
        if ((model) == PYRO_XY) {                                                   \
            if ((prec) == PYRO_FP64) VecOps<2, double>::call; else VecOps<2, float>::call; \
        } else {                                                                    \
            if ((prec) == PYRO_FP64) VecOps<3, double>::call; else VecOps<3, float>::call; \
        }                                                                           \
    } while (0)

cudaError_t vec_prepare(int model, int prec, const TileShape &t)
{
    if (model == PYRO_XY) return prec == PYRO_FP64 ? VecOps<2, double>::prepare(t, prec) : VecOps<2, float>::prepare(t, prec);
    return prec == PYRO_FP64 ? VecOps<3, double>::prepare(t, prec) : VecOps<3, float>::prepare(t, prec);
}

void vec_launch_init(int model, int prec, const Batch &B, int64_t nblocks, int random, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, init(B, nblocks, random, s));
}

// Phase p of a sweep: 0 local labelling, 1 boundary init, 2 boundary unite,
// 3 flip.
void vec_launch_phase(int p, int model, int prec, const Batch &B, int64_t ntiles, int64_t nblocks, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, phase(p, B, ntiles, prec, s));
    (void)nblocks;
}

void vec_launch_measure(int model, int prec, const Batch &B, int64_t nblocks, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, measure(B, nblocks, s));
}

}  // namespace pyro
