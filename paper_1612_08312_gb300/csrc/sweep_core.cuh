// sweep_core.cuh -- the model-independent parts of a Swendsen-Wang sweep:
// tile geometry, tile-local labelling in shared memory, the global union of
// tile-crossing clusters, and the resolution of every site to its cluster's
// canonical root.
//
// Bond bits of a cell: bit 12 f + k is bond k of FCC point f (k = 0..5 its
// "up" tetrahedron, k = 6..11 the "down" tetrahedron through site (f, 0)).
// Site bits: s = 4 f + mu.  Bond b = 48 c + 12 f + k of cell c.
#pragma once

#include "ccl.cuh"

namespace pyro {

// Position of the calling thread's cell in its tile and in the lattice.
struct TileCtx {
    int TX, TY, TZ, nt, L;
    int ox, oy, oz;
    int lx, ly, lz, t;
    int64_t cell;
    // local cell offset of a backward step along each axis (valid only if
    // the step stays in the tile), and whether it leaves the tile
    int dxm, dym, dzm;
    bool bx, by, bz;
};

__device__ __forceinline__ TileCtx tile_ctx(const Batch &B, const Rep &R, int64_t tile)
{
    TileCtx c;
    c.TX = B.TX;
    c.TY = B.TY;
    c.TZ = B.TZ;
    c.nt = B.TX * B.TY * B.TZ;
    c.L = R.L;
    c.ox = (int)(tile % R.ntx) * c.TX;
    c.oy = (int)((tile / R.ntx) % R.nty) * c.TY;
    c.oz = (int)(tile / ((int64_t)R.ntx * R.nty)) * c.TZ;
    c.t = threadIdx.x;
    c.lx = c.t % c.TX;
    c.ly = (c.t / c.TX) % c.TY;
    c.lz = c.t / (c.TX * c.TY);
    const int x = c.ox + c.lx, y = c.oy + c.ly, z = c.oz + c.lz;
    c.cell = (int64_t)x + (int64_t)c.L * ((int64_t)y + (int64_t)c.L * z);
    // a tile that spans a whole axis wraps onto itself along it
    c.bx = c.lx == 0 && c.TX != c.L;
    c.by = c.ly == 0 && c.TY != c.L;
    c.bz = c.lz == 0 && c.TZ != c.L;
    c.dxm = c.lx > 0 ? -1 : c.TX - 1;
    c.dym = c.ly > 0 ? -c.TX : (c.TY - 1) * c.TX;
    c.dzm = c.lz > 0 ? -c.TX * c.TY : (c.TZ - 1) * c.TX * c.TY;
    return c;
}

// Tile-local cell of a vertex whose cell is this cell stepped back along
// the axes of mask m (only meaningful if the vertex is inside the tile).
__device__ __forceinline__ int vertex_local_cell(const TileCtx &c, int m)
{
    return c.t + ((m & 1) ? c.dxm : 0) + ((m & 2) ? c.dym : 0) + ((m & 4) ? c.dzm : 0);
}

__device__ __forceinline__ bool vertex_inside(const TileCtx &c, int m)
{
    return !(((m & 1) && c.bx) || ((m & 2) && c.by) || ((m & 4) && c.bz));
}

__device__ __forceinline__ int wrap_back(int v, int L) { return v == 0 ? L - 1 : v - 1; }

// Global site index of vertex v of the down tetrahedron of FCC point f of
// cell (x, y, z).
__device__ __forceinline__ int down_vertex_global(int x, int y, int z, int L, int f, int v)
{
    const int m = down_mask(f, v);
    const int cx = (m & 1) ? wrap_back(x, L) : x;
    const int cy = (m & 2) ? wrap_back(y, L) : y;
    const int cz = (m & 4) ? wrap_back(z, L) : z;
    return 16 * (cx + L * (cy + L * cz)) + down_bit(f, v);
}

// The 16 flip bits of cell c: bits 16 c .. 16 c + 15 of the FLIP stream
// (bit i = bit i & 127 of call i >> 7).  One Philox call serves 8 cells;
// when the 8 cells are 8 consecutive lanes (TX a multiple of 8) the lane
// with lx % 8 == 0 draws it and shares it.
__device__ __forceinline__ uint32_t cell_flip_bits(const TileCtx &c, uint64_t seed, uint32_t sweep, uint32_t tag,
                                                   bool share)
{
    const uint64_t j = (uint64_t)c.cell >> 3;
    uint32_t word;
    const int wsel = (int)((c.cell & 7) >> 1);
    if (share) {
        // lanes present in this (possibly partial) warp of the block
        const int wbase = threadIdx.x & ~31;
        const int cnt = min(32, c.nt - wbase);
        const unsigned mask = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
        uint4 w = make_uint4(0, 0, 0, 0);
        if ((c.lx & 7) == 0) w = philox_call(seed, sweep, tag, j);
        const int leader = (threadIdx.x & 31) & ~7;
        w.x = __shfl_sync(mask, w.x, leader);
        w.y = __shfl_sync(mask, w.y, leader);
        w.z = __shfl_sync(mask, w.z, leader);
        w.w = __shfl_sync(mask, w.w, leader);
        word = word_of(w, wsel);
    } else {
        word = word_of(philox_call(seed, sweep, tag, j), wsel);
    }
    return (word >> (16 * (int)(c.cell & 1))) & 0xFFFFu;
}

// Bond decision from a 32-bit uniform assembled lazily: high half from the
// BOND call, low half (from the TIE call) only when the high halves tie.
// thr <= 2^32; the bond is active iff w < thr.
struct HalfCompare {
    uint32_t thi, tlo;
    bool all;
    __device__ __forceinline__ explicit HalfCompare(uint64_t thr)
        : thi((uint32_t)(thr >> 16)), tlo((uint32_t)(thr & 0xFFFFu)), all(thr >= (1ull << 32)) {}
};

// Shared-memory layout of the tile-local labelling, after the model's own
// staging area: labels (16 nt ints), the union-pair list (12 nt words) and
// its counter.
__host__ __device__ constexpr size_t core_smem_bytes(int nt) { return (size_t)16 * nt * 4 + (size_t)12 * nt * 4 + 16; }

// Tile-local labelling of one cell's sites given its 48 active-bond bits.
// Writes L16 (tile-local root of each site), F (flip bits) and, for face
// cells, dmask (union pairs leaving the tile).  Called by every thread of
// the block.
__device__ __forceinline__ void local_core(const TileCtx &c, const Rep &R, uint64_t act, uint32_t sweep,
                                           int *lab, uint32_t *plist, int *pcount)
{
    const int nt = c.nt;
    if (threadIdx.x == 0) *pcount = 0;
    // up tetrahedra: component minima in registers
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int rr[4];
        tet_components((uint32_t)(act >> (12 * f)) & 63u, rr);
#pragma unroll
        for (int v = 0; v < 4; ++v) lab[lslot(16 * c.t + 4 * f + v, nt)] = 16 * c.t + 4 * f + rr[v];
    }
    // down tetrahedra: union pairs (v, smallest vertex of v's component)
    uint32_t inpairs = 0, cross = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        int rr[4];
        tet_components((uint32_t)(act >> (12 * f + 6)) & 63u, rr);
#pragma unroll
        for (int v = 1; v < 4; ++v) {
            if (rr[v] == v) continue;
            const int k = pair_index(rr[v], v);
            const bool inside = vertex_inside(c, down_mask(f, rr[v])) && vertex_inside(c, down_mask(f, v));
            if (inside) inpairs |= 1u << (6 * f + k);
            else cross |= 1u << (6 * f + k);
        }
    }
    __syncthreads();  // labels initialised, counter cleared
    // append this cell's in-tile pairs to the block's list (the order of the
    // list does not change the final roots: they are cluster minima)
    const int n = __popc(inpairs);
    int base = n ? atomicAdd(pcount, n) : 0;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if ((inpairs >> (6 * f + k)) & 1u) {
                const int va = pair_a(k), vb = pair_b(k);
                const int a = 16 * vertex_local_cell(c, down_mask(f, va)) + down_bit(f, va);
                const int b = 16 * vertex_local_cell(c, down_mask(f, vb)) + down_bit(f, vb);
                plist[base++] = (uint32_t)a | ((uint32_t)b << 16);
            }
    __syncthreads();
    const int np = *pcount;
    bool ok = true;
    for (int e = threadIdx.x; e < np; e += nt) {
        const uint32_t pr = plist[e];
        ok &= sunite(lab, (int)(pr & 0xFFFFu), (int)(pr >> 16), nt);
    }
    if (!ok) atomicOr(&R.st->status, ST_NOCONVERGE);
    __syncthreads();
    // resolve to tile-local roots
    uint32_t packed[8];
#pragma unroll
    for (int s = 0; s < 16; s += 2) {
        const uint32_t r0 = (uint32_t)sfind(lab, 16 * c.t + s, nt);
        const uint32_t r1 = (uint32_t)sfind(lab, 16 * c.t + s + 1, nt);
        packed[s >> 1] = r0 | (r1 << 16);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(R.L16 + 16 * c.cell);
    dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    R.F[c.cell] = (uint16_t)cell_flip_bits(c, R.seed, sweep, TAG_FLIP, (c.TX & 7) == 0);
    if (c.lx == 0 || c.ly == 0 || c.lz == 0) R.dmask[c.cell] = cross;
}

// Global site index of the tile-local root stored for global site g.
__device__ __forceinline__ int crossing_root(const Rep &R, int TX, int TY, int TZ, int g)
{
    const int L = R.L;
    const int lr = R.L16[g] & 0x7FFF;
    const int cg = g >> 4;
    const int x = cg % L, y = (cg / L) % L, z = cg / (L * L);
    const int lc = lr >> 4;
    const int rx = (x / TX) * TX + lc % TX;
    const int ry = (y / TY) * TY + (lc / TX) % TY;
    const int rz = (z / TZ) * TZ + lc / (TX * TY);
    return 16 * (rx + L * (ry + L * rz)) + (lr & 15);
}

// Phase 1 (init) and 2 (unite) over the union pairs that leave a tile:
// init marks both endpoints' tile-local roots as crossing (bit 15 of their
// L16 entry) and makes each its own parent in P; unite merges them.
template <bool UNITE>
__global__ void __launch_bounds__(512) boundary_kernel(const __grid_constant__ Batch B)
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
        const int ga = down_vertex_global(x, y, z, L, f, pair_a(k));
        const int gb = down_vertex_global(x, y, z, L, f, pair_b(k));
        const int ra = crossing_root(R, TX, TY, TZ, ga);
        const int rb = crossing_root(R, TX, TY, TZ, gb);
        if (!UNITE) {
            R.P[ra] = ra;
            R.P[rb] = rb;
            unsigned *w = reinterpret_cast<unsigned *>(R.L16);
            atomicOr(w + (ra >> 1), 1u << (15 + 16 * (ra & 1)));
            atomicOr(w + (rb >> 1), 1u << (15 + 16 * (rb & 1)));
        } else {
            ok &= gunite(R.P, ra, rb);
        }
    }
    if (!ok) atomicOr(&R.st->status, ST_NOCONVERGE);
}

// Shared-memory bytes of the resolve stage: the tile's L16 entries (slot
// layout) and flip words.
__host__ __device__ constexpr size_t resolve_smem_bytes(int nt) { return (size_t)16 * nt * 2 + (size_t)nt * 2 + 16; }

// Resolve every site of the calling thread's cell to the global index of
// its cluster's root and the root's flip bit.  Stages the tile's L16 and F
// words in shared memory; roots of clusters that stay inside the tile are
// final, the others are looked up in P.  Called by every thread of the block.
__device__ __forceinline__ void resolve_cell(const TileCtx &c, const Rep &R, uint16_t *ls, uint16_t *fs, int root[16],
                                             uint32_t &flip)
{
    const int nt = c.nt;
    // stage: thread t loads cell t's 16 entries (32 contiguous bytes)
    const uint4 *src = reinterpret_cast<const uint4 *>(R.L16 + 16 * c.cell);
    const uint4 a0 = src[0], a1 = src[1];
    const uint32_t w[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int s = 0; s < 16; ++s) ls[lslot(16 * c.t + s, nt)] = (uint16_t)(w[s >> 1] >> (16 * (s & 1)));
    fs[c.t] = R.F[c.cell];
    __syncthreads();
    flip = 0;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int lr = (int)((w[s >> 1] >> (16 * (s & 1))) & 0x7FFFu);
        const int lc = lr >> 4;
        const int rx = c.ox + lc % c.TX, ry = c.oy + (lc / c.TX) % c.TY, rz = c.oz + lc / (c.TX * c.TY);
        int g = 16 * (rx + c.L * (ry + c.L * rz)) + (lr & 15);
        uint32_t fb;
        if (ls[lslot(lr, nt)] & 0x8000u) {
            g = root_of(R.P, g);
            fb = (R.F[g >> 4] >> (g & 15)) & 1u;
        } else {
            fb = (fs[lc] >> (lr & 15)) & 1u;
        }
        root[s] = g;
        flip |= fb << s;
    }
}

}  // namespace pyro
