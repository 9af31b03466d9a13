// ising.cu -- Swendsen-Wang sweep of the pyrochlore Ising model (Sec. 2).
//
// Spins are bit-packed, one uint16 per cubic cell (bit s of cell c is site
// 16 c + s; 1 means s = -1).  Every kernel runs over a Batch of one or more
// lattices, one CTA per tile of TX x TY x TZ cells, one thread per cell.
//
//   ising_local     reads its cell's spin word and those of the backward
//                   neighbour cells, forms the 48 bonds' antiparallel bits by
//                   shift-XOR, draws one Philox call per 16 bonds and
//                   compares its bytes with the threshold four at a time
//                   (a satisfied bond is active with p = 1 - exp(-2 beta J),
//                   the SW bond rule), then runs the tile-local labelling.
//   ising_flip      flips every site whose cluster's flip bit is set: the
//                   bit of its tile-local root, XOR that root's correction
//                   bit where the cluster crosses a tile face.
//   ising_measure   counts antiparallel bonds and -1 spins per tile, four
//                   cells per thread (exact integers; energy of Eq. 1,
//                   magnetisation of Eq. 2).
//   boundary_kernel unites the clusters that cross tile faces and sets the
//                   correction bits (all models).
//   labels_kernel   writes the canonical label of every site on demand.
#include <algorithm>

#include "sweep_core.cuh"

namespace pyro {

// Threads of a measurement block (a tile of up to 512 cells, four per thread).
constexpr int MEASURE_BLOCK = 128;

__global__ void __launch_bounds__(512) ising_local_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ __align__(16) int smem[];
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);
    const CoreSmem s = core_smem(smem, c.nt);
    const uint32_t sweep = (uint32_t)R.st->sweep;
    const uint64_t seed = R.seed;
    core_prologue(s);
    // the cell's spin word and those of the cells one step back along the
    // axes of each mask m (read straight from global memory, L1-cached)
    const uint16_t *spins = static_cast<const uint16_t *>(R.spins);
    uint32_t w[7];
    {
        const int L = c.L;
        const int x = c.ox + c.lx, y = c.oy + c.ly, z = c.oz + c.lz;
        const int xm = wrap_back(x, L), ym = wrap_back(y, L), zm = wrap_back(z, L);
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            const int cx = (m & 1) ? xm : x, cy = (m & 2) ? ym : y, cz = (m & 4) ? zm : z;
            w[m] = spins[(uint32_t)cx + (uint32_t)L * ((uint32_t)cy + (uint32_t)L * (uint32_t)cz)];
        }
    }
    __syncthreads();  // table and pair counters ready
    uint32_t anti[3];
    antiparallel_groups(w[0], down_word(w), anti[0], anti[1], anti[2]);
    uint32_t act[3];
    const ByteCompare bc(R.thr);
    if (bc.all || bc.none) {
#pragma unroll
        for (int g = 0; g < 3; ++g) act[g] = bc.all ? ~anti[g] & 0xFFFFu : 0u;
    } else {
        // bond 48 c + 16 g + 4 f + q: byte 4 f + q of BOND call 3 c + g; the
        // three calls are drawn together (independent chains interleave)
        uint4 wd[3];
#pragma unroll
        for (int g = 0; g < 3; ++g) wd[g] = philox_call(seed, sweep, TAG_BOND, 3 * (uint64_t)c.cell + g);
        const uint32_t t4 = bc.t8 * 0x01010101u;
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            const uint32_t sat = ~anti[g] & 0xFFFFu;
            const uint32_t ww[4] = {wd[g].x, wd[g].y, wd[g].z, wd[g].w};
            uint32_t a = 0;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                uint32_t nib = byte_flags_to_nibble(bytes_lt(ww[f], t4));
                uint32_t tie = byte_flags_to_nibble(bytes_eq(ww[f], t4)) & (sat >> (4 * f));
                while (tie) {  // top bytes equal: compare the low 24 bits
                    const int q = __ffs(tie) - 1;
                    tie &= tie - 1;
                    if (tie_bits(seed, sweep, c.cell, g, f, q) < bc.t24) nib |= 1u << q;
                }
                a |= nib << (4 * f);
            }
            act[g] = a & sat;
        }
    }
    local_core(c, R, s, act[0], act[1], act[2], sweep);
}

__global__ void __launch_bounds__(512) ising_flip_kernel(const __grid_constant__ Batch B)
{
    extern __shared__ __align__(16) int smem[];
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);
    const uint32_t flip = cell_flip_mask(c, R, smem);
    uint16_t *spins = static_cast<uint16_t *>(R.spins);
    spins[c.cell] = (uint16_t)((uint32_t)spins[c.cell] ^ flip);
}

// Canonical label (global index of the cluster root) of every site.
__global__ void __launch_bounds__(512) labels_kernel(const __grid_constant__ Batch B)
{
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);
    int root[16];
    uint32_t flip;
    resolve_cell(c, R, (uint32_t)R.st->last_epoch, root, flip);
    int4 *dst = reinterpret_cast<int4 *>(R.labels + 16 * c.cell);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_int4(root[4 * q], root[4 * q + 1], root[4 * q + 2], root[4 * q + 3]);
}

// Antiparallel bonds (48 per cell) and -1 spins: exact integer counts per
// tile, written to the tile's partial slot.
__global__ void __launch_bounds__(MEASURE_BLOCK) ising_measure_kernel(const __grid_constant__ Batch B)
{
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const TileCtx c = tile_ctx(B, R, blockIdx.x - B.tile_begin[r]);  // the tile's origin
    const uint16_t *spins = static_cast<const uint16_t *>(R.spins);
    const int L = c.L;
    unsigned anti = 0, ndown = 0;
    // up to four cells per thread: their 28 spin-word loads are independent
#pragma unroll 4
    for (int t = threadIdx.x; t < c.nt; t += blockDim.x) {
        const int x = c.ox + (t & (c.TX - 1)), y = c.oy + ((t >> c.lTX) & (c.TY - 1)), z = c.oz + (t >> (c.lTX + c.lTY));
        const int xm = wrap_back(x, L), ym = wrap_back(y, L), zm = wrap_back(z, L);
        uint32_t w[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            const int cx = (m & 1) ? xm : x, cy = (m & 2) ? ym : y, cz = (m & 4) ? zm : z;
            w[m] = spins[(uint32_t)cx + (uint32_t)L * ((uint32_t)cy + (uint32_t)L * (uint32_t)cz)];
        }
        uint32_t A, Bg, C;
        antiparallel_groups(w[0], down_word(w), A, Bg, C);
        anti += (unsigned)(__popc(A) + __popc(Bg) + __popc(C));
        ndown += (unsigned)__popc(w[0]);
    }
    anti = __reduce_add_sync(0xffffffffu, anti);  // blockDim is a multiple of 32
    ndown = __reduce_add_sync(0xffffffffu, ndown);
    __shared__ unsigned red[2][MEASURE_BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = anti;
        red[1][wid] = ndown;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sa = 0, sd = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
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

// Phase 1, over the face cells of every tile (one thread each): FLATTEN =
// false unites the clusters joined by the union pairs that leave the tile;
// FLATTEN = true then finds every crossing root's cluster root and, where
// the cluster root's flip bit differs from the crossing root's own, sets
// bit 14 of the crossing root's entry (a correction the flip kernel
// applies).  Model-independent: used by the n-vector sweeps too.
// Latency-bound chains of scattered loads: at most 32 registers, so that
// ten blocks of a 8 x 8 x 8 tile's 192 threads fit on an SM.
template <bool FLATTEN>
__global__ void __launch_bounds__(512, 4) boundary_kernel(const __grid_constant__ Batch B)
{
    // the block's crossing pairs, compacted so that every thread takes an
    // equal share: entry (face cell << 5) | (6 f + k)
    extern __shared__ uint16_t blist[];
    __shared__ int bcount;
    const int r = find_rep(B.tile_begin, B.R, blockIdx.x);
    const Rep &R = B.reps[r];
    const int nface = face_cells(B.TX, B.TY, B.TZ);
    const uint32_t tile = (uint32_t)(blockIdx.x - B.tile_begin[r]);
    const uint32_t txy = tile / (uint32_t)R.ntx;
    const int L = R.L;
    const int ox = (int)(tile - txy * (uint32_t)R.ntx) * B.TX;
    const int oy = (int)(txy % (uint32_t)R.nty) * B.TY;
    const int oz = (int)(txy / (uint32_t)R.nty) * B.TZ;
    if (threadIdx.x == 0) bcount = 0;
    __syncthreads();
    uint32_t todo = 0;
    if ((int)threadIdx.x < nface) {
        int lx, ly, lz;
        face_cell_coords(B, threadIdx.x, lx, ly, lz);
        todo = R.dmask[(int64_t)(ox + lx) + (int64_t)L * ((int64_t)(oy + ly) + (int64_t)L * (oz + lz))];
    }
    const int lane = threadIdx.x & 31;
    const int n = __popc(todo);
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int wtotal = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31 && wtotal) base = atomicAdd(&bcount, wtotal);
    int pos = __shfl_sync(0xffffffffu, base, 31) + incl - n;
    while (todo) {
        const int bit = __ffs(todo) - 1;
        todo &= todo - 1;
        blist[pos++] = (uint16_t)((threadIdx.x << 5) | bit);
    }
    __syncthreads();
    const int np = bcount;
    const uint32_t stamp = (uint32_t)R.st->epoch;
    unsigned long long *P = R.P;
    bool ok = true;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const uint32_t en = blist[i];
        int lx, ly, lz;
        face_cell_coords(B, (int)(en >> 5), lx, ly, lz);
        const int x = ox + lx, y = oy + ly, z = oz + lz;
        const int f = (int)(en & 31u) / 6, k = (int)(en & 31u) % 6;
        int g[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int v = e == 0 ? pair_a(k) : pair_b(k);
            const int m = down_mask(f, v);
            const int cx = (m & 1) ? wrap_back(x, L) : x;
            const int cy = (m & 2) ? wrap_back(y, L) : y;
            const int cz = (m & 4) ? wrap_back(z, L) : z;
            g[e] = crossing_root(R, B, cx, cy, cz, down_bit(f, v));
        }
        if (g[0] == g[1]) continue;  // both ends in one tile-local cluster
        if (!FLATTEN) {
            ok &= punite(P, g[0], g[1], stamp);
        } else {
            // both ends' cluster roots, walked together and read-only (all
            // unions are done and this pass writes no link, so the loads
            // may take the cached read-only path: many crossing roots share
            // one cluster root); a tile-local root that is not its
            // cluster's root gets the correction bit where the two flip
            // bits differ
            int rt[2] = {g[0], g[1]};
            unsigned long long v[2] = {__ldg(P + g[0]), __ldg(P + g[1])};
#pragma unroll 1
            for (int it = 0; it < (1 << 20) && (plinked(v[0], stamp) || plinked(v[1], stamp)); ++it) {
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (plinked(v[e], stamp)) rt[e] = (int)(uint32_t)v[e];
#pragma unroll
                for (int e = 0; e < 2; ++e)
                    if (plinked(v[e], stamp)) v[e] = __ldg(P + rt[e]);
            }
            unsigned *Lw = reinterpret_cast<unsigned *>(R.L16);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (rt[e] == g[e]) continue;
                const uint32_t d = (__ldg(R.F + (rt[e] >> 4)) >> (rt[e] & 15)) ^ (__ldg(R.F + (g[e] >> 4)) >> (g[e] & 15));
                if (d & 1u) {
                    const unsigned bitm = 1u << (14 + 16 * (g[e] & 1));
                    if (!(__ldcg(Lw + (g[e] >> 1)) & bitm)) atomicOr(Lw + (g[e] >> 1), bitm);
                }
            }
        }
    }
    if (!ok) atomicOr(&R.st->status, ST_NOCONVERGE);
}

// ------------------------------------------------------------ launchers --
cudaError_t ising_set_unite_bound(int bound) { return cudaMemcpyToSymbol(c_unite_bound, &bound, sizeof(int)); }

size_t ising_local_smem(const TileShape &t) { return core_smem_bytes(t.TX * t.TY * t.TZ); }

size_t resolve_smem(const TileShape &t) { return resolve_smem_bytes(t.TX * t.TY * t.TZ); }

cudaError_t ising_prepare(const TileShape &t)
{
    cudaError_t e = allow_dynamic_smem(ising_local_kernel, ising_local_smem(t));
    if (e == cudaSuccess) e = allow_dynamic_smem(ising_flip_kernel, resolve_smem(t));
    return e;
}

void ising_launch_init(const Batch &B, int64_t nblocks, int random, cudaStream_t s)
{
    ising_init_kernel<<<(unsigned)nblocks, CELL_BLOCK, 0, s>>>(B, random);
}

void launch_boundary(const Batch &B, int64_t ntiles, cudaStream_t s)
{
    const int nf = face_cells(B.TX, B.TY, B.TZ);
    const int threads = (nf + 31) & ~31;
    const size_t smem = (size_t)nf * 24 * sizeof(uint16_t);
    boundary_kernel<false><<<(unsigned)ntiles, threads, smem, s>>>(B);
    boundary_kernel<true><<<(unsigned)ntiles, threads, smem, s>>>(B);
}

void launch_labels(const Batch &B, int64_t ntiles, cudaStream_t s)
{
    labels_kernel<<<(unsigned)ntiles, B.TX * B.TY * B.TZ, 0, s>>>(B);
}

// Phase p of a sweep: 0 local labelling, 1 crossing unions, 2 flip.
void ising_launch_phase(int p, const Batch &B, int64_t ntiles, cudaStream_t s)
{
    const TileShape t{B.TX, B.TY, B.TZ};
    const int nt = B.TX * B.TY * B.TZ;
    if (p == 0) ising_local_kernel<<<(unsigned)ntiles, nt, ising_local_smem(t), s>>>(B);
    else if (p == 1) launch_boundary(B, ntiles, s);
    else ising_flip_kernel<<<(unsigned)ntiles, nt, resolve_smem(t), s>>>(B);
}

void ising_launch_measure(const Batch &B, int64_t ntiles, cudaStream_t s)
{
    const int nt = B.TX * B.TY * B.TZ;
    const int threads = std::min(MEASURE_BLOCK, std::max(32, ((nt + 3) / 4 + 31) & ~31));
    ising_measure_kernel<<<(unsigned)ntiles, threads, 0, s>>>(B);
}

}  // namespace pyro
