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
#include "nvec.cuh"
#include "sweep_core.cuh"

namespace pyro {

// 16 consecutive values of T (a cell's sites of one component, 64- or
// 128-byte aligned) to and from registers in 16-byte accesses.
template <typename T>
__device__ __forceinline__ void load16(const T *p, T out[16])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T)); ++k) {
        const uint4 w = q[k];
        memcpy(&out[k * 16 / (int)sizeof(T)], &w, 16);
    }
}

// 4 consecutive values of T (16-byte aligned) in 16-byte accesses.
template <typename T>
__device__ __forceinline__ void load4(const T *p, T out[4])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T)) / 4; ++k) {
        const uint4 w = q[k];
        memcpy(&out[k * 16 / (int)sizeof(T)], &w, 16);
    }
}

template <typename T>
__device__ __forceinline__ void store16(T *p, const T in[16])
{
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T)); ++k) {
        uint4 w;
        memcpy(&w, &in[k * 16 / (int)sizeof(T)], 16);
        q[k] = w;
    }
}

// The local kernel's staging area (the halo's projections, then the halo
// cells' first sites) is dead once the bonds are decided, before the
// labelling writes its labels and pair list: when it fits in their room
// (31 words a cell, the start of the core area) it shares it, which halves
// the shared memory of the FP32 kernels' common tiles.
__host__ __device__ constexpr size_t vec_stage_bytes(int TX, int TY, int TZ, size_t es)
{
    return (size_t)16 * halo_cells(TX, TY, TZ) * es + (size_t)halo_cells(TX, TY, TZ) * 4;
}

__host__ __device__ constexpr bool vec_stage_shared(int TX, int TY, int TZ, size_t es)
{
    return vec_stage_bytes(TX, TY, TZ, es) <= (size_t)31 * TX * TY * TZ * 4;
}

template <int NC, typename T>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) vec_local_kernel(const __grid_constant__ Batch B)
{
    using A = Ar<T>;
    extern __shared__ __align__(16) int smem[];
    const int rep = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[rep]);
    const CoreSmem sm = core_smem(smem, c.nt);
    const bool shared_stage = vec_stage_shared(c.TX, c.TY, c.TZ, sizeof(T));
    T *proj = reinterpret_cast<T *>(shared_stage ? reinterpret_cast<unsigned char *>(smem) : sm.stage);
    const T *spins = static_cast<const T *>(R.spins);
    const int64_t N = R.N;
    const uint32_t sweep = (uint32_t)R.st->sweep;
    const uint64_t seed = R.seed;
    core_prologue(sm);

    // the sweep's axis, drawn once per block (FP64 divides and square roots
    // run at a small fraction of the FP32 rate on this GPU)
    __shared__ double s_axis[3];
    if (threadIdx.x == 0) unit_vector_dev<NC>(seed, sweep, TAG_AXIS, 0, s_axis);
    __syncthreads();
    const T r[3] = {(T)s_axis[0], (T)s_axis[1], (T)s_axis[2]};

    // projections s_i . r of the tile's sites and the backward halo; each
    // halo cell's first site is found once (the halo's edges are not powers
    // of two, so this takes divisions) and shared.  Site-major layout (site s
    // of halo cell h at s nh + h): a warp's consecutive cells read
    // consecutive words (nh is odd, so the staging writes of one cell's 16
    // sites fall in 16 different banks too)
    const int nh = halo_cells(c.TX, c.TY, c.TZ);
    int *hbase = reinterpret_cast<int *>(proj + 16 * nh);
    for (int h = threadIdx.x; h < nh; h += blockDim.x)
        hbase[h] = (int)(16 * halo_cell(h, c.TX, c.TY, c.ox, c.oy, c.oz, c.L));
    __syncthreads();
    // four consecutive sites per thread, each component read in 16-byte
    // accesses (a cell's sites are 16-byte aligned in every plane)
    for (int idx = threadIdx.x; idx < 4 * nh; idx += blockDim.x) {
        const int h = idx >> 2, s0 = 4 * (idx & 3);
        const int64_t i0 = (int64_t)hbase[h] + s0;
        T v[NC][4];
#pragma unroll
        for (int k = 0; k < NC; ++k) load4(spins + k * N + i0, v[k]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T pr = A::mul(v[0][q], r[0]);  // in the order of project()
#pragma unroll
            for (int k = 1; k < NC; ++k) pr = A::add(pr, A::mul(v[k][q], r[k]));
            proj[(s0 + q) * nh + h] = pr;
        }
    }
    __syncthreads();

    const T K2 = (T)R.K2;
    uint32_t act[3] = {0, 0, 0};
    if (R.K2 > 0.0) {
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            T xb[16];
            uint32_t pos = 0;
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int va = slot_a(g, q), vb = slot_b(g, q);
                    T pa, pb;
                    if (slot_up(g, q)) {
                        pa = proj[(4 * f + va) * nh + halo_index(c, 0)];
                        pb = proj[(4 * f + vb) * nh + halo_index(c, 0)];
                    } else {
                        pa = proj[down_bit(f, va) * nh + halo_index(c, down_mask(f, va))];
                        pb = proj[down_bit(f, vb) * nh + halo_index(c, down_mask(f, vb))];
                    }
                    xb[4 * f + q] = A::mul(pa, pb);
                    pos |= (xb[4 * f + q] > (T)0 ? 1u : 0u) << (4 * f + q);
                }
            if (!pos) continue;
            const uint4 wd = philox_call(seed, sweep, TAG_BOND, 3 * (uint64_t)c.cell + g);
            const uint32_t ww[4] = {wd.x, wd.y, wd.z, wd.w};
            uint32_t a = 0;
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!((pos >> (4 * f + q)) & 1u)) continue;
                    const uint32_t byte = (ww[f] >> (8 * q)) & 0xFFu;
                    if (sizeof(T) == 4) {
                        // FP32: p = 1 - exp(-y), y = K2 x, exceeds (b + 1) / 256 (so the
                        // bond is on whatever the low bits) when y > -ln(1 - (b + 1) / 256),
                        // and stays below b / 256 (off) when y < -ln(1 - b / 256); the
                        // margins (1e-4 relative, 1e-6 absolute) exceed the errors of
                        // expm1f (1 ulp of p) and of __logf, so only bonds within them
                        // take the exact path below, with the same decision either way
                        const float y = (float)K2 * (float)xb[4 * f + q];
                        const float ylo = -__logf(1.0f - (float)byte * (1.0f / 256.0f));
                        const float yhi = -__logf(1.0f - (float)(byte + 1) * (1.0f / 256.0f));  // +inf for 255
                        if (y > yhi * 1.0001f + 1e-6f) {
                            a |= 1u << (4 * f + q);
                            continue;
                        }
                        if (y < ylo * 0.9999f - 1e-6f) continue;
                    }
                    const ByteCompare bc(prob_threshold(A::bond_p(K2, xb[4 * f + q])));
                    bool on = bc.all || byte < bc.t8;
                    if (!bc.all && !bc.none && byte == bc.t8) on = tie_bits(seed, sweep, c.cell, g, f, q) < bc.t24;
                    a |= (on && !bc.none ? 1u : 0u) << (4 * f + q);
                }
            act[g] = a;
        }
    }
    if (shared_stage) __syncthreads();  // the staging area is read no more: the labels may take it
    local_core(c, R, sm, act[0], act[1], act[2], sweep);
}

template <int NC, typename T>
__global__ void __launch_bounds__(512) vec_flip_kernel(const __grid_constant__ Batch B)
{
    using A = Ar<T>;
    extern __shared__ __align__(16) int smem[];
    const int rep = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[rep]);
    __shared__ double s_axis[3];
    if (threadIdx.x == 0) unit_vector_dev<NC>(R.seed, (uint32_t)R.st->sweep, TAG_AXIS, 0, s_axis);
    uint32_t flip = cell_flip_mask(c, R, smem);  // its barrier also publishes s_axis
    if (!flip) return;
    const T r[3] = {(T)s_axis[0], (T)s_axis[1], (T)s_axis[2]};
    T *spins = static_cast<T *>(R.spins);
    const int64_t N = R.N;
    if (NC * sizeof(T) > 16) {
        // FP64 Heisenberg: a cell's 48 doubles do not fit the registers;
        // site by site
        while (flip) {
            const int s = __ffs(flip) - 1;
            flip &= flip - 1;
            const int64_t i = 16 * c.cell + s;
            const T pr = project<NC, T>(spins, N, i, r);
            const T d2 = A::mul((T)2, pr);
            T t[3];
#pragma unroll
            for (int k = 0; k < NC; ++k) t[k] = A::sub(spins[k * N + i], A::mul(d2, r[k]));
            T q = A::mul(t[0], t[0]);
#pragma unroll
            for (int k = 1; k < NC; ++k) q = A::add(q, A::mul(t[k], t[k]));
            q = A::sqrt_(q);
#pragma unroll
            for (int k = 0; k < NC; ++k) spins[k * N + i] = A::div(t[k], q);
        }
        return;
    }
    // the cell's 16 sites of every component in registers (16-byte loads)
    T sv[NC][16];
#pragma unroll
    for (int k = 0; k < NC; ++k) load16(spins + k * N + 16 * c.cell, sv[k]);
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        if (!((flip >> s) & 1u)) continue;
        T pr = A::mul(sv[0][s], r[0]);  // the projection, in the order of project()
#pragma unroll
        for (int k = 1; k < NC; ++k) pr = A::add(pr, A::mul(sv[k][s], r[k]));
        const T d2 = A::mul((T)2, pr);
        T t[3];
#pragma unroll
        for (int k = 0; k < NC; ++k) t[k] = A::sub(sv[k][s], A::mul(d2, r[k]));
        T q = A::mul(t[0], t[0]);
#pragma unroll
        for (int k = 1; k < NC; ++k) q = A::add(q, A::mul(t[k], t[k]));
        q = A::sqrt_(q);
#pragma unroll
        for (int k = 0; k < NC; ++k) sv[k][s] = A::div(t[k], q);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) store16(spins + k * N + 16 * c.cell, sv[k]);
}

// Energy (Eq. 1) and magnetisation of the current configuration: every
// cell sums the 48 bonds it owns and its 16 spins (FP64 spins in FP64; FP32
// spins in FP32 within the cell, since FP64 adds and conversions run at a
// small fraction of the FP32 rate on this GPU), then in FP64; one partial
// (E, M_x, M_y, M_z) per tile, summed in a fixed order.
template <int NC, typename T>
__global__ void __launch_bounds__(512) vec_measure_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ __align__(16) int smem[];
    double *scratch = reinterpret_cast<double *>(smem);
    const int rep = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[rep];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[rep]);
    const int L = R.L;
    const int64_t N = R.N;
    const T *sp = static_cast<const T *>(R.spins);
    const int x = c.ox + c.lx, y = c.oy + c.ly, z = c.oz + c.lz;
    int64_t cb[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int cx = (m & 1) ? wrap_back(x, L) : x;
        const int cy = (m & 2) ? wrap_back(y, L) : y;
        const int cz = (m & 4) ? wrap_back(z, L) : z;
        cb[m] = 16 * ((int64_t)cx + (int64_t)L * ((int64_t)cy + (int64_t)L * cz));
    }
    // the cell's own 16 sites in registers (16-byte loads); the down
    // tetrahedra's vertices in backward cells are read from global memory
    T sv[NC][16];
#pragma unroll
    for (int k = 0; k < NC; ++k) load16(sp + k * N + cb[0], sv[k]);
    using Acc = T;  // the cell's own sums: the spins' precision
    Acc ec = (Acc)0, Mc[3] = {(Acc)0, (Acc)0, (Acc)0};
#pragma unroll
    for (int s = 0; s < 16; ++s)
#pragma unroll
        for (int k = 0; k < NC; ++k) Mc[k] += (Acc)sv[k][s];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int va = pair_a(k), vb = pair_b(k);
            T du = sv[0][4 * f + va] * sv[0][4 * f + vb];
#pragma unroll
            for (int q = 1; q < NC; ++q) du += sv[q][4 * f + va] * sv[q][4 * f + vb];
            const int ma = down_mask(f, va), mb = down_mask(f, vb);
            const int ba = down_bit(f, va), bb = down_bit(f, vb);
            T xa[3], xb[3];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                xa[q] = ma == 0 ? sv[q][ba] : sp[q * N + cb[ma] + ba];
                xb[q] = mb == 0 ? sv[q][bb] : sp[q * N + cb[mb] + bb];
            }
            T dd = xa[0] * xb[0];
#pragma unroll
            for (int q = 1; q < NC; ++q) dd += xa[q] * xb[q];
            ec += du + dd;
        }
    }
    const double e = (double)ec, M[3] = {(double)Mc[0], (double)Mc[1], (double)Mc[2]};
    double tot[4] = {e, M[0], M[1], M[2]};
    tile_sum4_f64(tot, c.nt, scratch);
    const double se = tot[0], s0 = tot[1], s1 = tot[2], s2 = tot[3];
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
cudaError_t vec_set_unite_bound(int bound) { return cudaMemcpyToSymbol(c_unite_bound, &bound, sizeof(int)); }

size_t resolve_smem(const TileShape &t);
void launch_boundary(const Batch &B, int64_t ntiles, cudaStream_t s);

size_t vec_local_smem(const TileShape &t, int prec)
{
    const size_t es = prec == PYRO_FP64 ? 8 : 4;
    const size_t core = core_smem_bytes(t.TX * t.TY * t.TZ);
    return vec_stage_shared(t.TX, t.TY, t.TZ, es) ? core : core + vec_stage_bytes(t.TX, t.TY, t.TZ, es);
}

static size_t vec_measure_smem(const TileShape &t) { return (size_t)4 * t.TX * t.TY * t.TZ * sizeof(double); }

template <int NC, typename T>
struct VecOps {
    static cudaError_t prepare(const TileShape &t, int prec)
    {
        cudaError_t e = allow_dynamic_smem(vec_local_kernel<NC, T>, vec_local_smem(t, prec));
        if (e == cudaSuccess) e = allow_dynamic_smem(vec_flip_kernel<NC, T>, resolve_smem(t));
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
        else if (p == 1) launch_boundary(B, ntiles, s);
        else vec_flip_kernel<NC, T><<<(unsigned)ntiles, nt, resolve_smem(t), s>>>(B);
    }
    static void measure(const Batch &B, int64_t ntiles, cudaStream_t s)
    {
        const TileShape t{B.TX, B.TY, B.TZ};
        vec_measure_kernel<NC, T><<<(unsigned)ntiles, B.TX * B.TY * B.TZ, vec_measure_smem(t), s>>>(B);
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

cudaError_t ising_prepare(const TileShape &t);

cudaError_t vec_prepare(int model, int prec, const TileShape &t)
{
    // the labels kernel (compiled with the Ising sweep) serves every model
    const cudaError_t e = ising_prepare(t);
    if (e != cudaSuccess) return e;
    if (model == PYRO_XY) return prec == PYRO_FP64 ? VecOps<2, double>::prepare(t, prec) : VecOps<2, float>::prepare(t, prec);
    return prec == PYRO_FP64 ? VecOps<3, double>::prepare(t, prec) : VecOps<3, float>::prepare(t, prec);
}

void vec_launch_init(int model, int prec, const Batch &B, int64_t nblocks, int random, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, init(B, nblocks, random, s));
}

// Phase p of a sweep: 0 local labelling, 1 crossing unions, 2 flip.
void vec_launch_phase(int p, int model, int prec, const Batch &B, int64_t ntiles, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, phase(p, B, ntiles, prec, s));
}

void vec_launch_measure(int model, int prec, const Batch &B, int64_t ntiles, cudaStream_t s)
{
    PYRO_VEC_DISPATCH(model, prec, measure(B, ntiles, s));
}

}  // namespace pyro
