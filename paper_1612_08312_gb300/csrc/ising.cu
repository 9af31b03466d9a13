// ising.cu -- Swendsen-Wang sweep of the pyrochlore Ising model (Sec. 2).
//
// Spins are bit-packed, one uint16 per cubic cell (bit s of cell c is site
// 16 c + s; 1 means s = -1).  Every kernel runs over a Batch of one or more
// lattices.  The Ising-specific kernels:
//
//   ising_local     one CTA per tile of TX x TY x TZ cells, one thread per
//                   cell.  Stages the tile's spin words plus a one-cell halo
//                   on the backward faces in shared memory and draws the
//                   random half-words of the satisfied bonds the cell owns:
//                   a satisfied bond is active with p = 1 - exp(-2 beta J)
//                   (SW bond activation).  Then the shared tile-local
//                   labelling (sweep_core.cuh).
//   ising_flip      resolves every site to its cluster root and flips the
//                   site iff the root's flip bit is set.
//   ising_measure   counts antiparallel bonds and -1 spins per block (exact
//                   integers; energy of Eq. 1, magnetisation of Eq. 2).
//   labels_kernel   writes the canonical label of every site on demand.
#include "sweep_core.cuh"

namespace pyro {

__host__ __device__ constexpr size_t ising_halo_bytes(int TX, int TY, int TZ)
{
    return (size_t)(TX + 1) * (TY + 1) * (TZ + 1) * sizeof(uint16_t);
}

__global__ void __launch_bounds__(512) ising_local_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ __align__(16) int smem[];
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);
    const int nt = c.nt, L = c.L;
    int *lab = smem;
    uint32_t *plist = reinterpret_cast<uint32_t *>(smem + 16 * nt);
    int *pcount = smem + 28 * nt;
    uint16_t *hs = reinterpret_cast<uint16_t *>(smem + 28 * nt + 4);
    const int HX = c.TX + 1, HY = c.TY + 1, HZ = c.TZ + 1;
    const uint16_t *spins = static_cast<const uint16_t *>(R.spins);
    const uint32_t sweep = (uint32_t)R.st->sweep;
    const uint64_t seed = R.seed;

    for (int h = threadIdx.x; h < HX * HY * HZ; h += blockDim.x) {
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        int gx = c.ox + hx - 1, gy = c.oy + hy - 1, gz = c.oz + hz - 1;
        gx += (gx < 0) ? L : 0;
        gy += (gy < 0) ? L : 0;
        gz += (gz < 0) ? L : 0;
        hs[h] = spins[(int64_t)gx + (int64_t)L * ((int64_t)gy + (int64_t)L * gz)];
    }
    __syncthreads();

    // spin words of this cell and its backward neighbours, by shift mask
    uint32_t w[7];
#pragma unroll
    for (int m = 0; m < 7; ++m)
        w[m] = hs[(c.lx + 1 - (m & 1)) + HX * ((c.ly + 1 - ((m >> 1) & 1)) + HY * (c.lz + 1 - ((m >> 2) & 1)))];

    uint64_t sat = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int va = pair_a(k), vb = pair_b(k);
            const uint32_t up = ((w[0] >> (4 * f + va)) ^ (w[0] >> (4 * f + vb))) & 1u;
            const uint32_t dn = ((w[down_mask(f, va)] >> down_bit(f, va)) ^ (w[down_mask(f, vb)] >> down_bit(f, vb))) & 1u;
            sat |= (uint64_t)(up ^ 1u) << (12 * f + k);
            sat |= (uint64_t)(dn ^ 1u) << (12 * f + 6 + k);
        }

    // Bond 48 c + j (j = 0..47) compares half j & 7 of BOND call 6 c + j / 8
    // (low half from TIE call 6 c + j / 8 on a tie) with the threshold.
    uint64_t act = 0;
    const HalfCompare hc(R.thr);
    if (hc.all) {
        act = sat;
    } else if (R.thr > 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const uint32_t byte = (uint32_t)(sat >> (8 * q)) & 0xFFu;
            if (!byte) continue;
            const uint64_t j = 6 * (uint64_t)c.cell + q;
            const uint4 wd = philox_call(seed, sweep, TAG_BOND, j);
            const uint32_t ww[4] = {wd.x, wd.y, wd.z, wd.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                if (!((byte >> h) & 1u)) continue;
                const uint32_t hi = (ww[h >> 1] >> (16 * (h & 1))) & 0xFFFFu;
                bool a = hi < hc.thi;
                if (hi == hc.thi) {
                    const uint4 wt = philox_call(seed, sweep, TAG_TIE, j);
                    a = ((word_of(wt, h >> 1) >> (16 * (h & 1))) & 0xFFFFu) < hc.tlo;
                }
                act |= (uint64_t)(a ? 1u : 0u) << (8 * q + h);
            }
        }
    }
    local_core(c, R, act, sweep, lab, plist, pcount);
}

__global__ void __launch_bounds__(512) ising_flip_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ __align__(16) int smem[];
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);
    uint16_t *ls = reinterpret_cast<uint16_t *>(smem);
    uint16_t *fs = ls + 16 * c.nt;
    int root[16];
    uint32_t flip;
    resolve_cell(c, R, ls, fs, root, flip);
    uint16_t *spins = static_cast<uint16_t *>(R.spins);
    spins[c.cell] = (uint16_t)((uint32_t)spins[c.cell] ^ flip);
}

// Canonical label (global index of the cluster root) of every site.
__global__ void __launch_bounds__(512) labels_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ __align__(16) int smem[];
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);
    uint16_t *ls = reinterpret_cast<uint16_t *>(smem);
    uint16_t *fs = ls + 16 * c.nt;
    int root[16];
    uint32_t flip;
    resolve_cell(c, R, ls, fs, root, flip);
    int4 *dst = reinterpret_cast<int4 *>(R.labels + 16 * c.cell);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_int4(root[4 * q], root[4 * q + 1], root[4 * q + 2], root[4 * q + 3]);
}

// Antiparallel bonds (48 per cell) and -1 spins, exact integer counts per
// block of CELL_BLOCK cells.
__global__ void __launch_bounds__(CELL_BLOCK) ising_measure_kernel(const __grid_constant__ Batch B)
{
    const int r = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const int64_t cell = (blockIdx.x - B.block_begin[r]) * CELL_BLOCK + threadIdx.x;
    unsigned long long anti = 0, ndown = 0;
    if (cell < R.ncells) {
        const int L = R.L;
        const uint16_t *spins = static_cast<const uint16_t *>(R.spins);
        const int x = (int)(cell % L), y = (int)((cell / L) % L), z = (int)(cell / ((int64_t)L * L));
        uint32_t w[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            const int cx = (m & 1) ? wrap_back(x, L) : x;
            const int cy = (m & 2) ? wrap_back(y, L) : y;
            const int cz = (m & 4) ? wrap_back(z, L) : z;
            w[m] = spins[(int64_t)cx + (int64_t)L * ((int64_t)cy + (int64_t)L * cz)];
        }
        uint32_t a = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int va = pair_a(k), vb = pair_b(k);
                a += ((w[0] >> (4 * f + va)) ^ (w[0] >> (4 * f + vb))) & 1u;
                a += ((w[down_mask(f, va)] >> down_bit(f, va)) ^ (w[down_mask(f, vb)] >> down_bit(f, vb))) & 1u;
            }
        anti = a;
        ndown = __popc(w[0]);
    }
    __shared__ unsigned long long red[2][CELL_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        anti += __shfl_xor_sync(0xffffffffu, anti, o);
        ndown += __shfl_xor_sync(0xffffffffu, ndown, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = anti;
        red[1][wid] = ndown;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sa = 0, sd = 0;
        for (int q = 0; q < CELL_BLOCK / 32; ++q) {
            sa += red[0][q];
            sd += red[1][q];
        }
        unsigned long long *o = reinterpret_cast<unsigned long long *>(B.partials + 4 * (int64_t)blockIdx.x);
        o[0] = sa;
        o[1] = sd;
    }
}

// Ordered or Philox-random start: site i is -1 iff bit i of the INIT stream
// (bit i & 127 of call i >> 7) is 1.
__global__ void __launch_bounds__(CELL_BLOCK) ising_init_kernel(const __grid_constant__ Batch B, int random)
{
    const int r = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const int64_t cell = (blockIdx.x - B.block_begin[r]) * CELL_BLOCK + threadIdx.x;
    if (cell >= R.ncells) return;
    uint32_t word = 0;
    if (random) {
        const uint4 wd = philox_call(R.seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)cell >> 3);
        word = (word_of(wd, (int)((cell & 7) >> 1)) >> (16 * (int)(cell & 1))) & 0xFFFFu;
    }
    static_cast<uint16_t *>(R.spins)[cell] = (uint16_t)word;
}

// ------------------------------------------------------------ launchers --
size_t ising_local_smem(const TileShape &t)
{
    const int nt = t.TX * t.TY * t.TZ;
    return core_smem_bytes(nt) + ising_halo_bytes(t.TX, t.TY, t.TZ);
}

size_t resolve_smem(const TileShape &t) { return resolve_smem_bytes(t.TX * t.TY * t.TZ); }

cudaError_t ising_prepare(const TileShape &t)
{
    cudaError_t e = cudaFuncSetAttribute(ising_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ising_local_smem(t));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ising_flip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)resolve_smem(t));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(labels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)resolve_smem(t));
    return e;
}

void ising_launch_init(const Batch &B, int64_t nblocks, int random, cudaStream_t s)
{
    ising_init_kernel<<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B, random);
}

void launch_boundary(int unite, const Batch &B, int64_t ntiles, cudaStream_t s)
{
    const int nt = B.TX * B.TY * B.TZ;
    if (unite) boundary_kernel<true><<<(unsigned)ntiles, nt, 0, s>>>(B);
    else boundary_kernel<false><<<(unsigned)ntiles, nt, 0, s>>>(B);
}

void launch_labels(const Batch &B, int64_t ntiles, cudaStream_t s)
{
    const TileShape t{B.TX, B.TY, B.TZ};
    labels_kernel<<<(unsigned)ntiles, B.TX * B.TY * B.TZ, resolve_smem(t), s>>>(B);
}

// Phase p of a sweep: 0 local labelling, 1 boundary init, 2 boundary unite,
// 3 flip.
void ising_launch_phase(int p, const Batch &B, int64_t ntiles, int64_t nblocks, cudaStream_t s)
{
    const TileShape t{B.TX, B.TY, B.TZ};
    const int nt = B.TX * B.TY * B.TZ;
    if (p == 0) ising_local_kernel<<<(unsigned)ntiles, nt, ising_local_smem(t), s>>>(B);
    else if (p == 1 || p == 2) launch_boundary(p == 2, B, ntiles, s);
    else ising_flip_kernel<<<(unsigned)ntiles, nt, resolve_smem(t), s>>>(B);
    (void)nblocks;
}

void ising_launch_measure(const Batch &B, int64_t nblocks, cudaStream_t s)
{
    ising_measure_kernel<<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B);
}

}  // namespace pyro
