// sweep_core.cuh -- the model-independent parts of a Swendsen-Wang sweep:
// tile geometry, tile-local labelling in shared memory, the global union of
// tile-crossing clusters, and the resolution of every site to its cluster's
// canonical root.
//
// Bonds of a cell.  Each of the cell's four FCC points f owns an "up"
// tetrahedron (its sites 4 f .. 4 f + 3) and a "down" tetrahedron (its
// site 4 f and three sites of backward neighbour cells).  The 48 bonds are
// kept as three 16-bit groups, bit 4 f + q of group g:
//   g = 0 (A): up pairs    q = 0 (0,1)  1 (1,2)  2 (2,3)  3 (0,3)
//   g = 1 (B): up (0,2), up (1,3), down (0,2), down (1,3)
//   g = 2 (C): down pairs  q = 0 (0,1)  1 (1,2)  2 (2,3)  3 (0,3)
// so that shift-XOR of a 16-bit spin word yields four bonds at once, and
// the bond with random-number id b = 48 c + 16 g + 4 f + q draws the top
// byte of its uniform from byte (b & 15) of BOND call b >> 4 = 3 c + g.
#pragma once

#include "ccl.cuh"

namespace pyro {

// Position of the calling thread's cell in its tile and in the lattice.
// Tile edges are powers of two (shifts, no divisions).
struct TileCtx {
    int TX, TY, TZ, lTX, lTY, nt, L;
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
    c.lTX = B.lTX;
    c.lTY = B.lTY;
    c.nt = B.TX * B.TY * B.TZ;
    c.L = R.L;
    // a lattice has fewer than 2^31 tiles (L <= 511): 32-bit divisions
    const uint32_t tl = (uint32_t)tile, ntx = (uint32_t)R.ntx, nty = (uint32_t)R.nty;
    const uint32_t txy = tl / ntx;
    c.ox = (int)(tl - txy * ntx) * c.TX;
    c.oy = (int)(txy % nty) * c.TY;
    c.oz = (int)(txy / nty) * c.TZ;
    c.t = threadIdx.x;
    c.lx = c.t & (c.TX - 1);
    c.ly = (c.t >> c.lTX) & (c.TY - 1);
    c.lz = c.t >> (c.lTX + c.lTY);
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

// Lanes of the calling thread's warp that exist in a block of nt threads.
__device__ __forceinline__ unsigned lanes_mask(int nt)
{
    const int cnt = min(32, nt - (int)(threadIdx.x & ~31u));
    return cnt >= 32 ? 0xffffffffu : ((1u << cnt) - 1u);
}

// Deterministic sums of four doubles over the block's nt threads: a fixed
// tree in shared memory (any nt), one barrier per level for all four;
// results valid in thread 0.  scratch holds 4 nt doubles.  (A warp-shuffle
// tree would add in FP64 on every lane at every level; FP64 adds are scarce
// on this GPU.)
__device__ __forceinline__ void tile_sum4_f64(double v[4], int nt, double *scratch)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) scratch[q * nt + t] = v[q];
    __syncthreads();
    int span = 1;
    while (span < nt) span <<= 1;
    for (int o = span >> 1; o > 0; o >>= 1) {
        if (t < o && t + o < nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) scratch[q * nt + t] = __dadd_rn(scratch[q * nt + t], scratch[q * nt + t + o]);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = scratch[q * nt];
}

// Tile-local cell of a vertex whose cell is this cell stepped back along
// the axes of mask m (only meaningful if the vertex is inside the tile).
__device__ __forceinline__ int vertex_local_cell(const TileCtx &c, int m)
{
    return c.t + ((m & 1) ? c.dxm : 0) + ((m & 2) ? c.dym : 0) + ((m & 4) ? c.dzm : 0);
}

__device__ __forceinline__ int wrap_back(int v, int L) { return v == 0 ? L - 1 : v - 1; }

// Cells of the backward halo staged by the tile kernels.
__host__ __device__ constexpr int halo_cells(int TX, int TY, int TZ) { return (TX + 1) * (TY + 1) * (TZ + 1); }

__device__ __forceinline__ int halo_index(const TileCtx &c, int m)
{
    const int HX = c.TX + 1, HY = c.TY + 1;
    return (c.lx + 1 - (m & 1)) + HX * ((c.ly + 1 - ((m >> 1) & 1)) + HY * (c.lz + 1 - ((m >> 2) & 1)));
}

// Global cell of halo entry h of the tile with origin (ox, oy, oz).
__device__ __forceinline__ int64_t halo_cell(int h, int TX, int TY, int ox, int oy, int oz, int L)
{
    const int HX = TX + 1, HY = TY + 1;
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    int gx = ox + hx - 1, gy = oy + hy - 1, gz = oz + hz - 1;
    gx += (gx < 0) ? L : 0;
    gy += (gy < 0) ? L : 0;
    gz += (gz < 0) ? L : 0;
    return (int64_t)gx + (int64_t)L * ((int64_t)gy + (int64_t)L * gz);
}

// ------------------------------------------------------ bond bit layout --
// Vertex pair of slot q of group g (see the header comment); up = whether
// the pair belongs to the up tetrahedron.
__host__ __device__ constexpr int slot_a(int g, int q) { return g == 1 ? (q & 1) : (q == 3 ? 0 : q); }
__host__ __device__ constexpr int slot_b(int g, int q) { return g == 1 ? (q & 1) + 2 : (q == 3 ? 3 : q + 1); }
__host__ __device__ constexpr bool slot_up(int g, int q) { return g == 0 || (g == 1 && q < 2); }

// Index into the tetrahedron table from a tetrahedron's bond bits: bits
// 0..3 pairs (0,1) (1,2) (2,3) (0,3), bits 4..5 pairs (0,2) (1,3).
__device__ __forceinline__ uint32_t up_tet_index(uint32_t A, uint32_t Bg, int f)
{
    return ((A >> (4 * f)) & 0xFu) | (((Bg >> (4 * f)) & 0x3u) << 4);
}
__device__ __forceinline__ uint32_t down_tet_index(uint32_t C, uint32_t Bg, int f)
{
    return ((C >> (4 * f)) & 0xFu) | (((Bg >> (4 * f + 2)) & 0x3u) << 4);
}

// Table entry of a tetrahedron with bond bits `idx` (order as above):
// 2 bits per vertex v = the smallest vertex connected to v.
__device__ __forceinline__ uint32_t tet_table_entry(uint32_t idx)
{
    int rr[4] = {0, 1, 2, 3};
    const int pa[6] = {0, 1, 2, 0, 0, 1};
    const int pb[6] = {1, 2, 3, 3, 2, 3};
#pragma unroll
    for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if ((idx >> k) & 1u) {
                const int m = min(rr[pa[k]], rr[pb[k]]);
                rr[pa[k]] = m;
                rr[pb[k]] = m;
            }
    return (uint32_t)(rr[0] | (rr[1] << 2) | (rr[2] << 4) | (rr[3] << 6));
}

// The four spins of the down tetrahedron of each FCC point f of a cell,
// gathered into one 16-bit word (bit 4 f + v = vertex v).  w[m] = spin word
// of the cell stepped back along the axes of mask m.
__device__ __forceinline__ uint32_t down_word(const uint32_t w[7])
{
    uint32_t D = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int v = 0; v < 4; ++v) D |= ((w[down_mask(f, v)] >> down_bit(f, v)) & 1u) << (4 * f + v);
    return D;
}

// Antiparallel bits of the three bond groups from the up and down spin
// words (shift-XOR within each nibble).
__device__ __forceinline__ void antiparallel_groups(uint32_t U, uint32_t D, uint32_t &A, uint32_t &Bg, uint32_t &C)
{
    const uint32_t u1 = U ^ (U >> 1), u2 = U ^ (U >> 2), u3 = U ^ (U >> 3);
    const uint32_t d1 = D ^ (D >> 1), d2 = D ^ (D >> 2), d3 = D ^ (D >> 3);
    A = (u1 & 0x7777u) | ((u3 & 0x1111u) << 3);
    Bg = (u2 & 0x3333u) | ((d2 & 0x3333u) << 2);
    C = (d1 & 0x7777u) | ((d3 & 0x1111u) << 3);
}

// Bytewise unsigned a < b: bit 7 of each byte of the result.
__device__ __forceinline__ uint32_t bytes_lt(uint32_t a, uint32_t b)
{
    const uint32_t d = (a | 0x80808080u) - (b & 0x7F7F7F7Fu);  // bit 7: low 7 bits of a >= those of b
    return ((~(a ^ b) & ~d) | (~a & b)) & 0x80808080u;
}

// Bytewise a == b: bit 7 of each byte.
__device__ __forceinline__ uint32_t bytes_eq(uint32_t a, uint32_t b)
{
    const uint32_t t = a ^ b;
    return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}

// Bit 7 of the four bytes -> four low bits.
__device__ __forceinline__ uint32_t byte_flags_to_nibble(uint32_t f) { return (((f >> 7) * 0x204081u) >> 21) & 0xFu; }

// Threshold of a bond: active iff its 32-bit uniform w < thr (thr <= 2^32).
// w's top byte comes from the BOND stream, its low 24 bits (only needed on
// a tie of the top bytes) from the TIE stream.
struct ByteCompare {
    uint32_t t8, t24;
    bool all, none;
    __device__ __forceinline__ explicit ByteCompare(uint64_t thr)
        : t8((uint32_t)(thr >> 24)), t24((uint32_t)(thr & 0xFFFFFFu)), all(thr >= (1ull << 32)), none(thr == 0) {}
};

// Low 24 bits of the TIE-stream word of bond id 48 c + 16 g + 4 f + q.
__device__ __forceinline__ uint32_t tie_bits(uint64_t seed, uint32_t sweep, int64_t cell, int g, int f, int q)
{
    const uint4 w = philox_call(seed, sweep, TAG_TIE, 12 * (uint64_t)cell + 4 * g + f);
    return word_of(w, q) & 0xFFFFFFu;
}

// The cell's 16 flip bits: bits 16 c .. 16 c + 15 of the FLIP stream (bit i
// = bit i & 127 of call i >> 7).  One Philox call serves 8 cells; when the
// 8 cells are 8 consecutive lanes (TX a multiple of 8) one lane draws it.
__device__ __forceinline__ uint32_t cell_flip_bits(const TileCtx &c, uint64_t seed, uint32_t sweep)
{
    const uint64_t j = (uint64_t)c.cell >> 3;
    const int wsel = (int)((c.cell & 7) >> 1);
    uint32_t word;
    if ((c.TX & 7) == 0) {
        const unsigned mask = lanes_mask(c.nt);
        uint4 w = make_uint4(0, 0, 0, 0);
        if ((c.lx & 7) == 0) w = philox_call(seed, sweep, TAG_FLIP, j);
        const int leader = (threadIdx.x & 31) & ~7;
        w.x = __shfl_sync(mask, w.x, leader);
        w.y = __shfl_sync(mask, w.y, leader);
        w.z = __shfl_sync(mask, w.z, leader);
        w.w = __shfl_sync(mask, w.w, leader);
        word = word_of(w, wsel);
    } else {
        word = word_of(philox_call(seed, sweep, TAG_FLIP, j), wsel);
    }
    return (word >> (16 * (int)(c.cell & 1))) & 0xFFFFu;
}

// --------------------------------------------------- tile-local labelling --
// Shared memory of the local kernels: labels (16 nt ints), union pairs
// (15 nt words), three pair counters and a pad word, tetrahedron table (64
// words); the model's staging area follows at the next 16-byte boundary
// (it holds doubles and 16-byte vectors).
__host__ __device__ constexpr int core_words(int nt) { return (31 * nt + 4 + 64 + 3) & ~3; }
__host__ __device__ constexpr size_t core_smem_bytes(int nt) { return (size_t)core_words(nt) * 4; }
static_assert(core_smem_bytes(1) % 16 == 0 && core_smem_bytes(2) % 16 == 0 && core_smem_bytes(8) % 16 == 0 &&
                  core_smem_bytes(512) % 16 == 0 && core_words(1) >= 31 + 68 && core_words(2) >= 62 + 68,
              "staging area must start on a 16-byte boundary after the core area");

// Union round of the down-tetrahedron pair k of FCC point f: the pair's two
// cells differ along the axes of m = mask(a) ^ mask(b).  Round 0: same cell
// or x only; round 1: y without z; round 2: z.  The rounds are separated by
// block barriers, so the trees grow row by row, then plane by plane; after
// the last round every component representative is pointed straight at
// its root.
__host__ __device__ constexpr int pair_round(int f, int k)
{
    return ((down_mask(f, pair_a(k)) ^ down_mask(f, pair_b(k))) & 4) ? 2
         : ((down_mask(f, pair_a(k)) ^ down_mask(f, pair_b(k))) & 2) ? 1 : 0;
}

// Pairs k of the down tetrahedron of f with a vertex whose cell is a
// backward step along axis d (bit k).
__host__ __device__ constexpr uint32_t pair_axis_mask(int f, int d)
{
    uint32_t m = 0;
    for (int k = 0; k < 6; ++k)
        if (((down_mask(f, pair_a(k)) | down_mask(f, pair_b(k))) >> d) & 1) m |= 1u << k;
    return m;
}

// Region of round r's pairs in the pair list: a cell has at most 7, 4 and
// 4 spanning pairs of rounds 0, 1 and 2 (at most 3 per tetrahedron, split
// over the rounds by the pair geometry).
__host__ __device__ constexpr int round_base(int r, int nt) { return r == 0 ? 0 : (r == 1 ? 7 * nt : 11 * nt); }

// Bit 6 f + k of the pair (0, f) of the down tetrahedron of f = 1..3 (pair
// index k = f - 1): its two vertices lie in the owning cell itself.
__host__ __device__ constexpr int own_pair_bit(int f) { return 7 * f - 1; }
__host__ __device__ constexpr uint32_t own_pair_bits() { return (1u << 6) | (1u << 13) | (1u << 20); }

__host__ __device__ constexpr uint32_t round_mask(int r)
{
    uint32_t m = 0;
    for (int f = 0; f < 4; ++f)
        for (int k = 0; k < 6; ++k)
            if (pair_round(f, k) == r) m |= 1u << (6 * f + k);
    return m;
}

struct CoreSmem {
    int *lab;
    uint32_t *plist;
    int *pcount;
    // tetrahedron table, by bond pattern: bits 0-7 the smallest vertex
    // connected to each vertex (2 bits each), bits 8-11 the component
    // representatives, bits 16-21 the spanning pairs (pair index k of
    // (smallest vertex, v) for every non-representative v)
    uint32_t *lut;
    unsigned char *stage;  // model staging area (16-byte aligned)
};

__device__ __forceinline__ CoreSmem core_smem(int *smem, int nt)
{
    CoreSmem s;
    s.lab = smem;
    s.plist = reinterpret_cast<uint32_t *>(smem + 16 * nt);
    s.pcount = smem + 31 * nt;  // three counters
    s.lut = reinterpret_cast<uint32_t *>(smem + 31 * nt + 4);
    s.stage = reinterpret_cast<unsigned char *>(smem + core_words(nt));
    return s;
}

// Called by every thread before the model's staging (covered by the same
// __syncthreads): clears the pair counters and fills the table.
__device__ __forceinline__ void core_prologue(const CoreSmem &s)
{
    if (threadIdx.x == 0) {  // the block may have fewer than three threads
        s.pcount[0] = 0;
        s.pcount[1] = 0;
        s.pcount[2] = 0;
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        const uint32_t e = tet_table_entry((uint32_t)i);
        uint32_t reps = 1, span = 0;
        for (int v = 1; v < 4; ++v) {
            const int rv = (int)((e >> (2 * v)) & 3u);
            if (rv == v) reps |= 1u << v;
            else span |= 1u << pair_index(rv, v);
        }
        s.lut[i] = e | (reps << 8) | (span << 16);
    }
}

// Tile-local labelling of one cell's sites from its active-bond groups.
// Writes L16 (tile-local root of each site), F (flip bits) and, for face
// cells, dmask (the union pairs that leave the tile: bit 6 f + k, k the
// pair index of (a, b) in the order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)).
// Called by every thread of the block after the staging barrier.
__device__ __forceinline__ void local_core(const TileCtx &c, const Rep &R, const CoreSmem &s, uint32_t A, uint32_t Bg,
                                           uint32_t C, uint32_t sweep)
{
    const int nt = c.nt;
    const uint32_t out = (c.bx ? 1u : 0u) | (c.by ? 2u : 0u) | (c.bz ? 4u : 0u);  // axes whose backward step leaves
    // the down tetrahedra's spanning pairs, split into those inside the
    // tile and those with a vertex across a backward tile face
    uint32_t inpairs = 0, cross = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const uint32_t span = (s.lut[down_tet_index(C, Bg, f)] >> 16) & 0x3Fu;
        const uint32_t leave = ((out & 1u) ? pair_axis_mask(f, 0) : 0u) | ((out & 2u) ? pair_axis_mask(f, 1) : 0u) |
                               ((out & 4u) ? pair_axis_mask(f, 2) : 0u);
        inpairs |= (span & ~leave) << (6 * f);
        cross |= (span & leave) << (6 * f);
    }
    // The pair (0, f) of the down tetrahedron of f = 1..3 joins site 4 f
    // (vertex 0 of up tetrahedron f) and site f (vertex f of up tetrahedron
    // 0), both in this cell: those three unions are made here, in the
    // initial labels, instead of in shared memory.
    const uint32_t own = inpairs & own_pair_bits();
    inpairs ^= own;
    uint32_t uptab[4];
    uint32_t reps = 0;  // bit 4 f + v: site is its component's representative
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        uptab[f] = s.lut[up_tet_index(A, Bg, f)];
        const bool joined = f > 0 && ((own >> own_pair_bit(f)) & 1u);
        reps |= (((uptab[f] >> 8) & 0xFu) & (joined ? ~1u : ~0u)) << (4 * f);
        const int rep0 = (int)((uptab[0] >> (2 * f)) & 3u);  // site f's representative in up tetrahedron 0
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int rv = (int)((uptab[f] >> (2 * v)) & 3u);
            s.lab[lslot(16 * c.t + 4 * f + v, nt)] = 16 * c.t + ((joined && rv == 0) ? rep0 : 4 * f + rv);
        }
    }
    // every round's pairs go to the round's own region of the pair list
    // before the first union
#pragma unroll
    for (int rnd = 0; rnd < 3; ++rnd) {
        const uint32_t mine = inpairs & round_mask(rnd);
        const int n = __popc(mine);
        int base = round_base(rnd, nt) + (n ? atomicAdd(s.pcount + rnd, n) : 0);
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (pair_round(f, k) == rnd && ((mine >> (6 * f + k)) & 1u)) {
                    const int va = pair_a(k), vb = pair_b(k);
                    const int a = 16 * vertex_local_cell(c, down_mask(f, va)) + down_bit(f, va);
                    const int b = 16 * vertex_local_cell(c, down_mask(f, vb)) + down_bit(f, vb);
                    s.plist[base++] = (uint32_t)a | ((uint32_t)b << 16);
                }
    }
    bool ok = true;
#pragma unroll
    for (int rnd = 0; rnd < 3; ++rnd) {
        __syncthreads();  // labels initialised and pairs listed / previous round's unions done
        const int np = s.pcount[rnd];
        const uint32_t *pl = s.plist + round_base(rnd, nt);
        for (int e = threadIdx.x; e < np; e += nt) {
            const uint32_t pr = pl[e];
            ok &= sunite(s.lab, (int)(pr & 0xFFFFu), (int)(pr >> 16), nt);
        }
    }
    __syncthreads();  // all unions done
    if (!ok) atomicOr(&R.st->status, ST_NOCONVERGE);
    // every representative's entry moves to its grandparent, all of them
    // together, until each points at its root (no unions any more, so the
    // entries only move up their trees; the work is spread evenly over the
    // threads, whatever the trees' depths)
    // A representative whose parent is a root (its entry is its own) is
    // done for good, since no entry changes any more but by these moves: it
    // leaves the thread's list, so later rounds only walk the deep ones.
    // After one such round the representatives left (on deeper chains)
    // are walked to their roots by their own threads, read-only, and pointed
    // at them: every entry on the way is an ancestor whatever the other
    // threads write meanwhile, so one barrier ends the whole resolution.
    volatile int *vl = s.lab;
    uint32_t todo = reps;
    bool done = false;
#pragma unroll 1
    for (int it = 0; it < 1 && !done; ++it) {
        int changed = 0;
        uint32_t pend = todo;
#pragma unroll 1
        while (pend) {
            const int q = __ffs(pend) - 1;
            pend &= pend - 1;
            const int x = 16 * c.t + q;
            const int p = vl[lslot(x, nt)];
            const int gp = vl[lslot(p, nt)];
            if (gp != p) {
                vl[lslot(x, nt)] = gp;
                changed = 1;
            } else {
                todo &= ~(1u << q);
            }
        }
        done = !__syncthreads_or(changed);  // the same for every thread
    }
    if (!done) {
        bool walked = true;
#pragma unroll 1
        while (todo) {
            const int q = __ffs(todo) - 1;
            todo &= todo - 1;
            const int x = 16 * c.t + q;
            int r = vl[lslot(x, nt)];
#pragma unroll 1
            for (int st = 0;; ++st) {
                const int p = vl[lslot(r, nt)];
                if (p == r) break;
                r = p;
                if (st == 16 * nt) {
                    walked = false;
                    break;
                }
            }
            vl[lslot(x, nt)] = r;
        }
        if (!walked) atomicOr(&R.st->status, ST_NOCONVERGE);
        __syncthreads();
    }
    // every site takes the root of its component's representative
    uint32_t packed[8];
    uint32_t root0[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool joined = f > 0 && ((own >> own_pair_bit(f)) & 1u);
        uint32_t root[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const uint32_t rv = (uptab[f] >> (2 * v)) & 3u;
            uint32_t r = 0;
#pragma unroll
            for (int u = 0; u < v; ++u)
                if (rv == (uint32_t)u) r = root[u];
            if (rv == (uint32_t)v) r = (v == 0 && joined) ? root0[f] : (uint32_t)vl[lslot(16 * c.t + 4 * f + v, nt)];
            root[v] = r;
        }
        if (f == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v) root0[v] = root[v];
        }
        packed[2 * f] = root[0] | (root[1] << 16);
        packed[2 * f + 1] = root[2] | (root[3] << 16);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(R.L16 + 16 * c.cell);
    dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    R.F[c.cell] = (uint16_t)cell_flip_bits(c, R.seed, sweep);
    if (c.lx == 0 || c.ly == 0 || c.lz == 0) R.dmask[c.cell] = cross;
}

// ------------------------------------------------ crossing clusters (HBM) --
// P64[x] = (stamp << 32) | parent.  An entry whose stamp is not the current
// sweep's is a root (left over from an earlier sweep), so P64 needs no
// clearing: linking a root is a compare-and-swap from the value just read.
// The larger root is always hung under the smaller one, so a cluster's root
// stays its minimum site index.
__device__ __forceinline__ bool plinked(unsigned long long v, uint32_t stamp) { return (uint32_t)(v >> 32) == stamp; }

// One find step with path splitting: x (entry v, a current link) moves to
// its parent, whose entry is returned in v; x's entry is pointed at its
// grandparent if that is a current link.  One dependent load per level.
__device__ __forceinline__ void pstep(unsigned long long *P, int &x, unsigned long long &v, uint32_t stamp)
{
    const int p = (int)(uint32_t)v;
    const unsigned long long gv = __ldcg(P + p);
    if (plinked(gv, stamp)) __stcg(P + x, gv);
    x = p;
    v = gv;
}

// Union of the crossing clusters of a and b.  Both finds walk in lockstep
// (their loads overlap); a root is linked by a compare-and-swap from the
// entry value its walk ended on.  Returns false if the bound was hit.
__device__ __forceinline__ bool punite(unsigned long long *P, int a, int b, uint32_t stamp)
{
    unsigned long long va = __ldcg(P + a), vb = __ldcg(P + b);
#pragma unroll 1
    for (int it = 0; it < (1 << 20); ++it) {
        const bool la = plinked(va, stamp), lb = plinked(vb, stamp);
        if (la || lb) {
            if (la) pstep(P, a, va, stamp);
            if (lb) pstep(P, b, vb, stamp);
            continue;
        }
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
            const unsigned long long tv = va;
            va = vb;
            vb = tv;
        }
        const unsigned long long nv = ((unsigned long long)stamp << 32) | (uint32_t)a;
        const unsigned long long old = atomicCAS(P + b, vb, nv);
        if (old == vb) return true;
        vb = old;  // b was linked meanwhile: walk on from its new entry
    }
    return false;
}

// Root of x after all unions of the sweep (plain cached loads).
__device__ __forceinline__ int proot(const unsigned long long *P, int x, uint32_t stamp)
{
#pragma unroll 1
    for (int it = 0; it < (1 << 20); ++it) {
        const unsigned long long v = P[x];
        if ((uint32_t)(v >> 32) != stamp) return x;
        x = (int)(uint32_t)v;
    }
    return x;
}

// Global site index of the tile-local root stored for the site (cell (x, y,
// z), offset s) with power-of-two tile edges.
__device__ __forceinline__ int crossing_root(const Rep &R, const Batch &B, int x, int y, int z, int s)
{
    const int L = R.L;
    const int lr = R.L16[16 * ((int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z)) + s] & 0x1FFF;
    const int lc = lr >> 4;
    const int rx = (x & ~(B.TX - 1)) + (lc & (B.TX - 1));
    const int ry = (y & ~(B.TY - 1)) + ((lc >> B.lTX) & (B.TY - 1));
    const int rz = (z & ~(B.TZ - 1)) + (lc >> (B.lTX + B.lTY));
    return 16 * (rx + L * (ry + L * rz)) + (lr & 15);
}

// Shared-memory bytes of the flip stage: one corrected flip word per cell.
__host__ __device__ constexpr size_t resolve_smem_bytes(int nt) { return (size_t)nt * 2 + 16; }

// Resolve every site of the calling thread's cell to the global index of
// its cluster's root and the root's flip bit.  The tile-local root of each
// site comes from L16; a tile-local root that was linked in P this sweep
// (stamp) belongs to a crossing cluster and its links are followed to the
// cluster root.  Called by every thread of the block.
__device__ __forceinline__ void resolve_cell(const TileCtx &c, const Rep &R, uint32_t stamp, int root[16],
                                             uint32_t &flip)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(R.L16 + 16 * c.cell);
    const uint4 a0 = src[0], a1 = src[1];
    const uint32_t w[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    flip = 0;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int lr = (int)((w[s >> 1] >> (16 * (s & 1))) & 0x1FFFu);
        const int lc = lr >> 4;
        const int rx = c.ox + (lc & (c.TX - 1));
        const int ry = c.oy + ((lc >> c.lTX) & (c.TY - 1));
        const int rz = c.oz + (lc >> (c.lTX + c.lTY));
        const int g = proot(R.P, 16 * (rx + c.L * (ry + c.L * rz)) + (lr & 15), stamp);
        root[s] = g;
        flip |= ((R.F[g >> 4] >> (g & 15)) & 1u) << s;
    }
}

// Flip mask of the calling thread's cell (bit s = site 16 c + s flips).  A
// site flips with its tile-local root's bit of F, corrected by bit 14 of
// that root's L16 entry when its cluster crosses a tile face and the
// cluster root's flip bit differs (written by the crossing pass).  Each
// thread folds its own cell's correction bits into its F word, so the tile
// shares one 16-bit word per cell in shared memory.  No global lookups.
// Called by every thread of the block.
__device__ __forceinline__ uint32_t cell_flip_mask(const TileCtx &c, const Rep &R, int *smem)
{
    uint16_t *fx = reinterpret_cast<uint16_t *>(smem);
    const uint4 *src = reinterpret_cast<const uint4 *>(R.L16 + 16 * c.cell);
    const uint4 a0 = src[0], a1 = src[1];
    const uint32_t w[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    uint32_t corr = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) corr |= (((w[i] >> 14) & 1u) | ((w[i] >> 29) & 2u)) << (2 * i);
    fx[c.t] = (uint16_t)(R.F[c.cell] ^ corr);
    __syncthreads();
    uint32_t flip = 0;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        const int lr = (int)((w[s >> 1] >> (16 * (s & 1))) & 0x1FFFu);
        flip |= ((fx[lr >> 4] >> (lr & 15)) & 1u) << s;
    }
    return flip;
}

// ------------------------------------------------------- face-cell grid --
// Cells of a tile with lx == 0, ly == 0 or lz == 0 (the cells that own the
// tetrahedra leaving the tile), enumerated compactly: the lz == 0 plane,
// then for each lz > 0 the row ly == 0 and the column lx == 0.
__host__ __device__ constexpr int face_cells(int TX, int TY, int TZ) { return TX * TY * TZ - (TX - 1) * (TY - 1) * (TZ - 1); }

__device__ __forceinline__ void face_cell_coords(const Batch &B, int i, int &lx, int &ly, int &lz)
{
    const int plane = B.TX * B.TY;
    if (i < plane) {
        lz = 0;
        ly = i >> B.lTX;
        lx = i & (B.TX - 1);
        return;
    }
    const int per = B.TX + B.TY - 1;
    const int j = i - plane;
    lz = 1 + j / per;
    const int k = j - (lz - 1) * per;
    if (k < B.TX) {
        ly = 0;
        lx = k;
    } else {
        ly = k - B.TX + 1;
        lx = 0;
    }
}

}  // namespace pyro
