// ising.cu -- Swendsen-Wang sweep of the pyrochlore Ising model (Sec. 2).
//
// Spins are bit-packed, one uint16 per cubic cell (bit s of cell c is site
// 16 c + s; 1 means s = -1).  Every kernel runs over a Batch of one or more
// lattices.  A sweep is:
//
//   ising_local     one CTA per tile of TX x TY x TZ cells, one thread per
//                   cell.  Stages the tile's spin words plus a one-cell halo
//                   on the backward faces in shared memory, draws the Philox
//                   word of every satisfied bond the cell owns (SW bond
//                   activation, p = 1 - exp(-2 beta J)), unites the four
//                   sites of each up tetrahedron in registers and the down-
//                   tetrahedron bonds inside the tile in shared memory, and
//                   writes P[i] = global index of i's tile-local root, the
//                   flip bits of the tile-local roots, and the active bonds
//                   that leave the tile.
//   ising_boundary  unites in HBM (atomicMin) the clusters joined by the
//                   tile-crossing bonds.
//   ising_flip      follows every site to its root (= minimum site index of
//                   its cluster, the canonical label), flips the site iff the
//                   root's flip bit is set, and stores the label.
//   ising_measure   counts antiparallel bonds and -1 spins per block (exact
//                   integers; energy of Eq. 1, magnetisation of Eq. 2).
//   measure_accumulate (engine.cu) turns the counts into E, m^2, m^4.
#include "ccl.cuh"

namespace pyro {

// Tile-local cell coordinate stepped back along one axis, or -1 if that
// leaves the tile (a tile that spans the whole axis wraps onto itself).
__device__ __forceinline__ int local_back(int l, int T, int L)
{
    if (l > 0) return l - 1;
    return (T == L) ? T - 1 : -1;
}

__device__ __forceinline__ int wrap_back(int c, int L) { return c == 0 ? L - 1 : c - 1; }

__global__ void __launch_bounds__(1024) ising_local_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ int smem[];
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const uint16_t *spins = static_cast<const uint16_t *>(R.spins);
    const int L = R.L;
    const int TX = B.TX, TY = B.TY, TZ = B.TZ;
    const int nt = TX * TY * TZ;
    int *lab = smem;
    uint16_t *hs = reinterpret_cast<uint16_t *>(smem + 16 * nt);
    const int HX = TX + 1, HY = TY + 1, HZ = TZ + 1;

    const int64_t tile = blockIdx.x - B.tile_begin[r];
    const int ox = (int)(tile % R.ntx) * TX;
    const int oy = (int)((tile / R.ntx) % R.nty) * TY;
    const int oz = (int)(tile / ((int64_t)R.ntx * R.nty)) * TZ;
    const uint32_t sweep = (uint32_t)R.st->sweep;
    const uint64_t seed = R.seed, thr = R.thr;

    // Stage the tile's spin words and the backward halo.
    for (int h = threadIdx.x; h < HX * HY * HZ; h += blockDim.x) {
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        int gx = ox + hx - 1, gy = oy + hy - 1, gz = oz + hz - 1;
        gx += (gx < 0) ? L : 0;
        gy += (gy < 0) ? L : 0;
        gz += (gz < 0) ? L : 0;
        hs[h] = spins[(int64_t)gx + (int64_t)L * ((int64_t)gy + (int64_t)L * gz)];
    }
    __syncthreads();

    const int t = threadIdx.x;
    const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
    const int x = ox + lx, y = oy + ly, z = oz + lz;
    const int64_t cell = (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z);

    // Spin words of this cell and its backward neighbours, by shift mask.
    uint32_t w[7];
#pragma unroll
    for (int m = 0; m < 7; ++m)
        w[m] = hs[(lx + 1 - (m & 1)) + HX * ((ly + 1 - ((m >> 1) & 1)) + HY * (lz + 1 - ((m >> 2) & 1)))];

    uint32_t dn_act = 0;  // 6 bits per f: active down-tetrahedron bonds
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        uint32_t su[4], sd[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            su[v] = (w[0] >> (4 * f + v)) & 1u;
            sd[v] = (w[down_mask(f, v)] >> down_bit(f, v)) & 1u;
        }
        uint32_t sat = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            sat |= (su[pair_a(k)] == su[pair_b(k)] ? 1u : 0u) << k;
            sat |= (sd[pair_a(k)] == sd[pair_b(k)] ? 1u : 0u) << (6 + k);
        }
        // Bond b = 12 r + k uses word k & 3 of call 3 r + k / 4 (r = 4 c + f).
        uint32_t act = 0;
        if (thr >= (1ull << 32)) {
            act = sat;
        } else if (thr > 0) {
            const uint64_t rf = 4 * (uint64_t)cell + f;
#pragma unroll
            for (int g = 0; g < 3; ++g) {
                if ((sat >> (4 * g)) & 0xFu) {
                    const uint4 wd = philox_call(seed, sweep, TAG_BOND, 3 * rf + g);
                    const uint32_t ww[4] = {wd.x, wd.y, wd.z, wd.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        act |= (((sat >> (4 * g + q)) & 1u) && (uint64_t)ww[q] < thr ? 1u : 0u) << (4 * g + q);
                }
            }
        }
        // Up tetrahedron: component minima of its four sites, in registers.
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

    // Down-tetrahedron bonds: unite inside the tile, defer the rest.
    const int lxb = local_back(lx, TX, L), lyb = local_back(ly, TY, L), lzb = local_back(lz, TZ, L);
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

    // Resolve to tile-local roots; write the global indices of those roots.
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

    // Flip bits of the tile-local roots: site 16 c + 4 f + mu takes word mu
    // of flip call 4 c + f.
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

// Global unions for the active bonds that cross a tile face.
__global__ void __launch_bounds__(1024) boundary_kernel(const __grid_constant__ Batch B)
{
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const int TX = B.TX, TY = B.TY, TZ = B.TZ, L = R.L;
    const int t = threadIdx.x;
    const int lx = t % TX, ly = (t / TX) % TY, lz = t / (TX * TY);
    if (!(lx == 0 || ly == 0 || lz == 0)) return;
    const int64_t tile = blockIdx.x - B.tile_begin[r];
    const int x = (int)(tile % R.ntx) * TX + lx;
    const int y = (int)((tile / R.ntx) % R.nty) * TY + ly;
    const int z = (int)(tile / ((int64_t)R.ntx * R.nty)) * TZ + lz;
    const int64_t cell = (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z);
    uint32_t todo = R.dmask[cell];
    bool ok = true;
    while (todo) {
        const int bit = __ffs(todo) - 1;
        todo &= todo - 1;
        const int f = bit / 6, k = bit % 6;
        int g[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int v = e == 0 ? pair_a(k) : pair_b(k);
            const int m = down_mask(f, v);
            const int cx = (m & 1) ? wrap_back(x, L) : x;
            const int cy = (m & 2) ? wrap_back(y, L) : y;
            const int cz = (m & 4) ? wrap_back(z, L) : z;
            g[e] = 16 * (cx + L * (cy + L * cz)) + down_bit(f, v);
        }
        ok &= gunite(R.P, g[0], g[1]);
    }
    if (!ok) atomicOr(&R.st->status, ST_NOCONVERGE);
}

__global__ void __launch_bounds__(CELL_BLOCK) ising_flip_kernel(const __grid_constant__ Batch B)
{
    const int r = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const int64_t cell = (blockIdx.x - B.block_begin[r]) * CELL_BLOCK + threadIdx.x;
    if (cell >= R.ncells) return;
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
    uint32_t flip = 0;
    bool changed = false;
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
    uint16_t *spins = static_cast<uint16_t *>(R.spins);
    spins[cell] = (uint16_t)((uint32_t)spins[cell] ^ flip);
}

// Antiparallel bonds (48 per cell: the two tetrahedra of each of its four
// FCC points) and -1 spins, exact integer counts per block.
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

// Ordered or Philox-random start: site i is -1 iff bit 31 of word i of the
// INIT stream is 1 (call i >> 2 = 4 c + f, word mu).
__global__ void __launch_bounds__(CELL_BLOCK) ising_init_kernel(const __grid_constant__ Batch B, int random)
{
    const int r = find_rep(B.block_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const int64_t cell = (blockIdx.x - B.block_begin[r]) * CELL_BLOCK + threadIdx.x;
    if (cell >= R.ncells) return;
    uint32_t word = 0;
    if (random) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const uint4 wd = philox_call(R.seed, INIT_SWEEP_FIELD, TAG_INIT, 4 * (uint64_t)cell + f);
            word |= ((wd.x >> 31) | ((wd.y >> 31) << 1) | ((wd.z >> 31) << 2) | ((wd.w >> 31) << 3)) << (4 * f);
        }
    }
    static_cast<uint16_t *>(R.spins)[cell] = (uint16_t)word;
}

// ------------------------------------------------------------ launchers --
size_t ising_local_smem(const TileShape &t)
{
    const int nt = t.TX * t.TY * t.TZ;
    return (size_t)16 * nt * sizeof(int) + (size_t)(t.TX + 1) * (t.TY + 1) * (t.TZ + 1) * sizeof(uint16_t);
}

cudaError_t ising_prepare(const TileShape &t)
{
    return cudaFuncSetAttribute(ising_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ising_local_smem(t));
}

void ising_launch_init(const Batch &B, int64_t nblocks, int random, cudaStream_t s)
{
    ising_init_kernel<<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B, random);
}

// Phase p of a sweep: 0 local labelling, 1 boundary unions, 2 flip.
void ising_launch_phase(int p, const Batch &B, int64_t ntiles, int64_t nblocks, cudaStream_t s)
{
    const TileShape t{B.TX, B.TY, B.TZ};
    const int nt = B.TX * B.TY * B.TZ;
    if (p == 0) ising_local_kernel<<<(unsigned)ntiles, nt, ising_local_smem(t), s>>>(B);
    else if (p == 1) boundary_kernel<<<(unsigned)ntiles, nt, 0, s>>>(B);
    else ising_flip_kernel<<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B);
}

void launch_boundary(const Batch &B, int64_t ntiles, cudaStream_t s)
{
    boundary_kernel<<<(unsigned)ntiles, B.TX * B.TY * B.TZ, 0, s>>>(B);
}

void ising_launch_measure(const Batch &B, int64_t nblocks, cudaStream_t s)
{
    ising_measure_kernel<<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B);
}

}  // namespace pyro
