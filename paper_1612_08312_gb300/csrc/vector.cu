// vector.cu -- Swendsen-Wang sweep of the pyrochlore XY (n = 2) and
// Heisenberg (n = 3) models with Wolff's embedded-cluster construction
// (Sec. 2): per sweep one random unit axis r; the projections p_i = s_i.r
// define an Ising model with couplings J p_i p_j; bonds with p_i p_j > 0 are
// activated with probability 1 - exp(-2 beta J p_i p_j); flipped clusters
// reflect their spins, s -> s - 2 (s.r) r.
//
// Spins are stored as n component planes of N values of T (float or
// double).  The FP64 path uses explicitly rounded IEEE operations in the
// same order as the definition, so projections, reflections and the axis
// are bit-identical to a straightforward FP64 evaluation without fused
// multiply-add.  The FP32 path stores and updates spins in float; its
// measurements are accumulated in FP64.
//
// Kernels (each over a Batch of lattices): vec_local (projections of the
// tile + halo staged in shared memory, bond activation, tile-local
// labelling), the global union of tile-crossing bonds (boundary_kernel,
// shared with the Ising sweep), vec_flip (root, flip, reflection) and
// vec_measure (E and M per block in FP64).
#include "ccl.cuh"

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
    static __device__ __forceinline__ double uword(uint32_t w)
    {
        return __dmul_rn(__dadd_rn((double)w, 0.5), 2.3283064365386962890625e-10);
    }
};

template <>
struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float div(float a, float b) { return a / b; }
    static __device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
    static __device__ __forceinline__ float bond_p(float K2, float x) { return -expm1f(-(K2 * x)); }
    static __device__ __forceinline__ float uword(uint32_t w)
    {
        return ((float)w + 0.5f) * 2.3283064365386962890625e-10f;
    }
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

template <int NC, typename T>
__global__ void __launch_bounds__(512) vec_local_kernel(const __grid_constant__ Batch B)
{
    using A = Ar<T>;
    extern __shared__ int smem[];
    const int rep = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const T *spins = static_cast<const T *>(R.spins);
    const int L = R.L;
    const int64_t N = R.N;
    const int TX = B.TX, TY = B.TY, TZ = B.TZ;
    const int nt = TX * TY * TZ;
    const int HX = TX + 1, HY = TY + 1, HZ = TZ + 1;
    int *lab = smem;
    T *proj = reinterpret_cast<T *>(smem + 16 * nt + ((16 * nt) & 1));
    const uint32_t sweep = (uint32_t)R.st->sweep;
    const uint64_t seed = R.seed;

    double rd[3];
    unit_vector_dev<NC>(seed, sweep, TAG_AXIS, 0, rd);
    const T r[3] = {(T)rd[0], (T)rd[1], (T)rd[2]};

    const int64_t tile = blockIdx.x - B.tile_begin[rep];
    const int ox = (int)(tile % R.ntx) * TX;
    const int oy = (int)((tile / R.ntx) % R.nty) * TY;
    const int oz = (int)(tile / ((int64_t)R.ntx * R.nty)) * TZ;

    for (int idx = threadIdx.x; idx < 16 * HX * HY * HZ; idx += blockDim.x) {
        const int h = idx >> 4, s = idx & 15;
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        int gx = ox + hx - 1, gy = oy + hy - 1, gz = oz + hz - 1;
        gx += (gx < 0) ? L : 0;
        gy += (gy < 0) ? L : 0;
        gz += (gz < 0) ? L : 0;
        const int64_t i = 16 * ((int64_t)gx + (int64_t)L * ((int64_t)gy + (int64_t)L * gz)) + s;
        proj[idx] = project<NC, T>(spins, N, i, r);
    }
    __syncthreads();

    const int t = threadIdx.x;
    const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
    const int x = ox + lx, y = oy + ly, z = oz + lz;
    const int64_t cell = (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z);
    const T K2 = (T)R.K2;

    uint32_t dn_act = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        T pu[4], pd[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            pu[v] = proj[16 * ((lx + 1) + HX * ((ly + 1) + HY * (lz + 1))) + 4 * f + v];
            const int m = down_mask(f, v);
            const int hidx = (lx + 1 - (m & 1)) + HX * ((ly + 1 - ((m >> 1) & 1)) + HY * (lz + 1 - ((m >> 2) & 1)));
            pd[v] = proj[16 * hidx + down_bit(f, v)];
        }
        T xb[12];
        uint32_t pos = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            xb[k] = A::mul(pu[pair_a(k)], pu[pair_b(k)]);
            xb[6 + k] = A::mul(pd[pair_a(k)], pd[pair_b(k)]);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) pos |= (xb[k] > (T)0 ? 1u : 0u) << k;

        uint32_t act = 0;
        if (R.K2 > 0.0) {
            const uint64_t rr_fcc = 4 * (uint64_t)cell + f;
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                if ((pos >> (4 * g)) & 0xFu) {
                    const uint4 wd = philox_call(seed, sweep, TAG_BOND, 3 * rr_fcc + g);
                    const uint32_t ww[4] = {wd.x, wd.y, wd.z, wd.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = 4 * g + q;
                        if ((pos >> k) & 1u) {
                            const T p = A::bond_p(K2, xb[k]);
                            act |= (A::uword(ww[q]) < p ? 1u : 0u) << k;
                        }
                    }
                }
            }
        }

        int rr[4] = {0, 1, 2, 3};
#pragma unroll
        for (int pass = 0; pass < 3; ++pass)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if ((act >> k) & 1u) {
                    const int m = min(rr[pair_a(k)], rr[pair_b(k)]);
                    rr[pair_a(k)] = m;
                    rr[pair_b(k)] = m;
                }
#pragma unroll
        for (int v = 0; v < 4; ++v) lab[16 * t + 4 * f + v] = 16 * t + 4 * f + rr[v];
        dn_act |= ((act >> 6) & 63u) << (6 * f);
    }
    __syncthreads();

    const int lxb = lx > 0 ? lx - 1 : (TX == L ? TX - 1 : -1);
    const int lyb = ly > 0 ? ly - 1 : (TY == L ? TY - 1 : -1);
    const int lzb = lz > 0 ? lz - 1 : (TZ == L ? TZ - 1 : -1);
    uint32_t cross = 0;
    bool ok = true;
    uint32_t todo = dn_act;
    while (todo) {
        const int bit = __ffs(todo) - 1;
        todo &= todo - 1;
        const int f = bit / 6, k = bit % 6;
        int loc[2];
        bool inside = true;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int v = e == 0 ? pair_a(k) : pair_b(k);
            const int m = down_mask(f, v);
            const int cx = (m & 1) ? lxb : lx, cy = (m & 2) ? lyb : ly, cz = (m & 4) ? lzb : lz;
            if (cx < 0 || cy < 0 || cz < 0) inside = false;
            loc[e] = 16 * (cx + TX * (cy + TY * cz)) + down_bit(f, v);
        }
        if (inside) ok &= sunite(lab, loc[0], loc[1]);
        else cross |= 1u << bit;
    }
    if (lx == 0 || ly == 0 || lz == 0) R.dmask[cell] = cross;
    if (!ok) atomicOr(&R.st->status, ST_NOCONVERGE);
    __syncthreads();

    int root_g[16];
    uint32_t is_root = 0;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int me = 16 * t + s;
        const int rl = sfind(lab, me);
        is_root |= (rl == me ? 1u : 0u) << s;
        const int rc = rl >> 4;
        const int rx = ox + rc % TX, ry = oy + (rc / TX) % TY, rz = oz + rc / (TX * TY);
        root_g[s] = 16 * (rx + L * (ry + L * rz)) + (rl & 15);
    }
    int4 *P4 = reinterpret_cast<int4 *>(R.P + 16 * cell);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        P4[q] = make_int4(root_g[4 * q], root_g[4 * q + 1], root_g[4 * q + 2], root_g[4 * q + 3]);
    uint32_t fb = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if ((is_root >> (4 * f)) & 0xFu) {
            const uint4 wd = philox_call(seed, sweep, TAG_FLIP, 4 * (uint64_t)cell + f);
            fb |= ((wd.x >> 31) | ((wd.y >> 31) << 1) | ((wd.z >> 31) << 2) | ((wd.w >> 31) << 3)) << (4 * f);
        }
    }
    R.F[cell] = (uint16_t)(fb & is_root);
}

template <int NC, typename T>
__global__ void __launch_bounds__(CELL_BLOCK) vec_flip_kernel(const __grid_constant__ Batch B)
{
    using A = Ar<T>;
    const int rep = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const int64_t cell = (blockIdx.x - B.block_begin[rep]) * CELL_BLOCK + threadIdx.x;
    if (cell >= R.ncells) return;
    double rd[3];
    unit_vector_dev<NC>(R.seed, (uint32_t)R.st->sweep, TAG_AXIS, 0, rd);
    const T r[3] = {(T)rd[0], (T)rd[1], (T)rd[2]};
    T *spins = static_cast<T *>(R.spins);
    const int32_t *P = R.P;
    int4 *P4 = reinterpret_cast<int4 *>(R.P + 16 * cell);
    int p[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int4 v = P4[q];
        p[4 * q] = v.x;
        p[4 * q + 1] = v.y;
        p[4 * q + 2] = v.z;
        p[4 * q + 3] = v.w;
    }
    bool changed = false;
    uint32_t flip = 0;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int rt = root_of(P, p[s]);
        flip |= ((uint32_t)(R.F[rt >> 4] >> (rt & 15)) & 1u) << s;
        changed |= (rt != p[s]);
        p[s] = rt;
    }
    if (changed) {
#pragma unroll
        for (int q = 0; q < 4; ++q) P4[q] = make_int4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
    }
    const int64_t N = R.N;
    while (flip) {
        const int s = __ffs(flip) - 1;
        flip &= flip - 1;
        const int64_t i = 16 * cell + s;
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
size_t vec_local_smem(const TileShape &t, int prec)
{
    const int nt = t.TX * t.TY * t.TZ;
    const size_t es = prec == PYRO_FP64 ? 8 : 4;
    return (size_t)(16 * nt + ((16 * nt) & 1)) * sizeof(int) +
           (size_t)16 * (t.TX + 1) * (t.TY + 1) * (t.TZ + 1) * es;
}

void launch_boundary(const Batch &B, int64_t ntiles, cudaStream_t s);

template <int NC, typename T>
struct VecOps {
    static cudaError_t prepare(const TileShape &t, int prec)
    {
        return cudaFuncSetAttribute(vec_local_kernel<NC, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)vec_local_smem(t, prec));
    }
    static void init(const Batch &B, int64_t nblocks, int random, cudaStream_t s)
    {
        vec_init_kernel<NC, T><<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B, random);
    }
    static void phase(int p, const Batch &B, int64_t ntiles, int64_t nblocks, int prec, cudaStream_t s)
    {
        const TileShape t{B.TX, B.TY, B.TZ};
        if (p == 0) vec_local_kernel<NC, T><<<(unsigned)ntiles, B.TX * B.TY * B.TZ, vec_local_smem(t, prec), s>>>(B);
        else if (p == 1) launch_boundary(B, ntiles, s);
        else vec_flip_kernel<NC, T><<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B);
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

// Phase p of a sweep: 0 local labelling, 1 boundary unions, 2 flip.
void vec_launch_phase(int p, int model, int prec, const Batch &B, int64_t ntiles, int64_t nblocks, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, phase(p, B, ntiles, nblocks, prec, s));
}

void vec_launch_measure(int model, int prec, const Batch &B, int64_t nblocks, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, measure(B, nblocks, s));
}

}  // namespace pyro
