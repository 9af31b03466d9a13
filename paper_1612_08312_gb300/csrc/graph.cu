// graph.cu -- Swendsen-Wang sweep on a generic lattice: an explicit list of
// nearest-neighbour bonds (Sec. 2: the program needs only each site's
// neighbour table), the simple-cubic lattice with implicit bonds (Sec. 3.4,
// the comparison lattice of Eq. 5-6), either one optionally diluted by a
// site mask and a bond mask (Sec. 4).  Ising (n = 1) and the embedded-
// cluster n-vector models (n = 2, 3), conventions as in include/pyro.h.
//
// A sweep is four launches (five for n > 1):
//   graph_proj   (n > 1) the sweep's axis r and every projection s_i . r;
//   graph_bond   one thread per 16 consecutive bond ids: one Philox call
//                gives their top bytes, the tie call is drawn only when a
//                top byte equals the threshold's; active bonds are united
//                in a global union-find array (atomicMin, larger root under
//                the smaller, so a finished cluster's root is its minimum
//                site, the canonical label).  The same threads draw the
//                sweep's flip bits, 128 sites per call;
//   graph_flip   one thread per site: root, canonical label, flip
//                (Ising: negate; n > 1: reflect and renormalise), and the
//                identity labels of the next sweep's array (two arrays
//                alternate, so no separate reset launch is needed);
//   graph_measure / graph_accumulate   E over present bonds and M over
//                occupied sites, per block in a fixed order, then one block
//                forms E, m^2, m^4 and adds them to the Neumaier sums.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "engine.h"
#include "nvec.cuh"

namespace pyro {

struct GraphDev {
    int64_t N, NB, nocc;
    int L;     // simple-cubic edge; 0 = explicit bond list
    int nc;    // spin components
    const int32_t *bi, *bj;
    const uint32_t *present;  // bond bit set (bond mask and both ends occupied), or null
    const uint32_t *occ;      // site bit set, or null
    void *spins;              // Ising int8 +-1; n > 1 nc planes of N values of T
    int32_t *lab, *lab_next;
    uint32_t *fb;             // flip bits, 4 words per 128 sites
    void *proj;               // n > 1: projections s_i . r (T)
    double *axis;             // n > 1: the sweep's axis
    double *partials;         // 4 per measurement block
    DevStats *st;
    uint64_t seed, thr;
    double K2, J;
};

constexpr int GB_THREADS = 256;

// Simple cubic: coordinates of site s and its neighbour one step along
// +axis d (32-bit arithmetic: N < 2^31).
__device__ __forceinline__ void sc_coords(int L, int s, int &x, int &y, int &z)
{
    const unsigned us = (unsigned)s, uL = (unsigned)L, t = us / uL;
    x = (int)(us - t * uL);
    z = (int)(t / uL);
    y = (int)(t - (unsigned)z * uL);
}

__device__ __forceinline__ int sc_next(int L, int s, int x, int y, int z, int d)
{
    if (d == 0) return x + 1 == L ? s - x : s + 1;
    if (d == 1) return y + 1 == L ? s - y * L : s + L;
    return z + 1 == L ? s - z * L * L : s + L * L;
}

// Sites joined by bond e.
__device__ __forceinline__ void bond_ends(const GraphDev &G, int64_t e, int &i, int &j)
{
    if (G.L) {
        const int64_t s = e / 3;
        int x, y, z;
        sc_coords(G.L, (int)s, x, y, z);
        i = (int)s;
        j = sc_next(G.L, i, x, y, z, (int)(e - 3 * s));
    } else {
        i = G.bi[e];
        j = G.bj[e];
    }
}

__device__ __forceinline__ bool bit_of(const uint32_t *set, int64_t k) { return (set[k >> 5] >> (k & 31)) & 1u; }

// Union of the clusters of a and b in the global array (path halving in
// both finds).  False if the union's iteration bound was hit.
__device__ bool gunite(int32_t *lab, int a, int b)
{
    volatile int32_t *vl = lab;
    const int bound = c_unite_bound;
    int pa = vl[a], pb = vl[b];
#pragma unroll 1
    for (int it = 0; it < bound; ++it) {
#pragma unroll 1
        for (int st = 0; (pa != a || pb != b) && st < (1 << 20); ++st) {
            if (pa != a) {
                const int g = vl[pa];
                if (g != pa) vl[a] = g;
                a = pa;
                pa = g;
            }
            if (pb != b) {
                const int g = vl[pb];
                if (g != pb) vl[b] = g;
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
        const int old = atomicMin(&lab[b], a);
        if (old == b) return true;
        // b had been linked meanwhile: unite a with its new parent
        b = old;
        pa = vl[a];
        pb = vl[b];
    }
    return false;
}

template <int NC, typename T>
__global__ void __launch_bounds__(GB_THREADS) graph_init_kernel(const __grid_constant__ GraphDev G, int random)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.N) return;
    G.lab[i] = (int32_t)i;
    G.lab_next[i] = (int32_t)i;
    if (NC == 1) {
        int neg = 0;
        if (random) {
            const uint4 w = philox_call(G.seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i >> 7);
            neg = (word_of(w, (int)((i & 127) >> 5)) >> (i & 31)) & 1;
        }
        static_cast<int8_t *>(G.spins)[i] = neg ? -1 : 1;
    } else {
        double r[3] = {1.0, 0.0, 0.0};
        if (random) unit_vector_dev<NC>(G.seed, INIT_SWEEP_FIELD, TAG_INIT, (uint64_t)i << 8, r);
#pragma unroll
        for (int k = 0; k < NC; ++k) static_cast<T *>(G.spins)[k * G.N + i] = (T)r[k];
    }
}

template <int NC, typename T>
__global__ void __launch_bounds__(GB_THREADS) graph_proj_kernel(const __grid_constant__ GraphDev G)
{
    __shared__ double rs[3];
    if (threadIdx.x == 0) {
        unit_vector_dev<NC>(G.seed, (uint32_t)G.st->sweep, TAG_AXIS, 0, rs);
        if (blockIdx.x == 0)
            for (int k = 0; k < 3; ++k) G.axis[k] = rs[k];
    }
    __syncthreads();
    const T r[3] = {(T)rs[0], (T)rs[1], (T)rs[2]};
    const T *sp = static_cast<const T *>(G.spins);
    T *proj = static_cast<T *>(G.proj);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.N; i += (int64_t)gridDim.x * blockDim.x)
        proj[i] = project<NC, T>(sp, G.N, i, r);
}

// Thread c takes the 16 bonds 16 c .. 16 c + 15 (one BOND call) and draws
// the FLIP call c.  (One bond per lane with the words passed by shuffles was
// measured slower: a warp's lanes then unite the bonds of the same few sites
// at once.)
template <int NC, typename T>
__global__ void __launch_bounds__(GB_THREADS) graph_bond_kernel(const __grid_constant__ GraphDev G)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t sweep = (uint32_t)G.st->sweep;
    if (128 * c < G.N) reinterpret_cast<uint4 *>(G.fb)[c] = philox_call(G.seed, sweep, TAG_FLIP, (uint64_t)c);
    const int64_t e0 = 16 * c;
    if (e0 >= G.NB) return;
    const uint4 w = philox_call(G.seed, sweep, TAG_BOND, (uint64_t)c);
    const int nq = (int)(G.NB - e0 < 16 ? G.NB - e0 : 16);
    uint32_t pres = 0xFFFFu;
    if (G.present) pres = (G.present[e0 >> 5] >> (e0 & 31)) & 0xFFFFu;
    bool ok = true;
    // simple cubic: bond 3 s + d, walked incrementally from the chunk's first
    int s = 0, d = 0, x = 0, y = 0, z = 0;
    if (G.L) {
        const uint64_t s0 = (uint64_t)e0 / 3u;
        s = (int)s0;
        d = (int)((uint64_t)e0 - 3u * s0);
        sc_coords(G.L, s, x, y, z);
    }
#pragma unroll 1
    for (int q = 0; q < nq; ++q) {
        if (G.L && q > 0 && ++d == 3) {
            d = 0;
            ++s;
            if (++x == G.L) {
                x = 0;
                if (++y == G.L) {
                    y = 0;
                    ++z;
                }
            }
        }
        if (!((pres >> q) & 1u)) continue;
        const int64_t e = e0 + q;
        int i, j;
        if (G.L) {
            i = s;
            j = sc_next(G.L, s, x, y, z, d);
        } else {
            i = G.bi[e];
            j = G.bj[e];
        }
        uint64_t thr;
        if (NC == 1) {
            const int8_t *sp = static_cast<const int8_t *>(G.spins);
            if (sp[i] != sp[j]) continue;
            thr = G.thr;
        } else {
            const T *p = static_cast<const T *>(G.proj);
            const T xp = Ar<T>::mul(p[i], p[j]);
            if (!(xp > (T)0)) continue;
            thr = prob_threshold(Ar<T>::bond_p((T)G.K2, xp));
        }
        const uint64_t byte = (word_of(w, q >> 2) >> (8 * (q & 3))) & 0xFFu;
        const uint64_t hi = thr >> 24;
        bool act = byte < hi;
        if (byte == hi) {
            const uint4 t = philox_call(G.seed, sweep, TAG_TIE, (uint64_t)e >> 2);
            act = (word_of(t, (int)(e & 3)) & 0xFFFFFFu) < (uint32_t)(thr & 0xFFFFFFu);
        }
        if (act && !gunite(G.lab, i, j)) ok = false;
    }
    if (!ok) atomicOr(&G.st->status, ST_NOCONVERGE);
}

template <int NC, typename T>
__global__ void __launch_bounds__(GB_THREADS) graph_flip_kernel(const __grid_constant__ GraphDev G)
{
    using A = Ar<T>;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G.N) return;
    const volatile int32_t *vl = G.lab;
    int r = vl[i];
    int steps = 0;
#pragma unroll 1
    for (;;) {
        const int p = vl[r];
        if (p == r) break;
        r = p;
        if (++steps > UF_MAX_ITERS) {
            atomicOr(&G.st->status, ST_NOCONVERGE);
            break;
        }
    }
    G.lab_next[i] = (int32_t)i;
    G.lab[i] = r;
    if (G.occ && !bit_of(G.occ, i)) return;
    if (!bit_of(G.fb, r)) return;
    if (NC == 1) {
        int8_t *s = static_cast<int8_t *>(G.spins);
        s[i] = (int8_t)(-s[i]);
    } else {
        T *sp = static_cast<T *>(G.spins);
        const T rr[3] = {(T)G.axis[0], (T)G.axis[1], (T)G.axis[2]};
        const T d2 = A::mul((T)2, static_cast<const T *>(G.proj)[i]);
        T sv[3];
#pragma unroll
        for (int k = 0; k < NC; ++k) sv[k] = A::sub(sp[k * G.N + i], A::mul(d2, rr[k]));
        T q = A::mul(sv[0], sv[0]);
#pragma unroll
        for (int k = 1; k < NC; ++k) q = A::add(q, A::mul(sv[k], sv[k]));
        q = A::sqrt_(q);
#pragma unroll
        for (int k = 0; k < NC; ++k) sp[k * G.N + i] = A::div(sv[k], q);
    }
}

// Per block: sum over present bonds of s_i . s_j and the occupied sites'
// magnetisation components, in a fixed order (grid-stride, then a fixed
// shuffle tree).  Ising sums are integers, exact in FP64.
template <int NC, typename T>
__global__ void __launch_bounds__(GB_THREADS) graph_measure_kernel(const __grid_constant__ GraphDev G)
{
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (NC == 1) {
        const int8_t *s = static_cast<const int8_t *>(G.spins);
        long long e = 0, m = 0;
        for (int64_t i = t0; i < G.N; i += stride)
            if (!G.occ || bit_of(G.occ, i)) m += s[i];
        if (G.L) {
            for (int64_t i = t0; i < G.N; i += stride) {
                int x, y, z;
                sc_coords(G.L, (int)i, x, y, z);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (G.present && !bit_of(G.present, 3 * i + d)) continue;
                    e += s[i] == s[sc_next(G.L, (int)i, x, y, z, d)] ? 1 : -1;
                }
            }
        } else {
            for (int64_t b = t0; b < G.NB; b += stride) {
                if (G.present && !bit_of(G.present, b)) continue;
                e += s[G.bi[b]] == s[G.bj[b]] ? 1 : -1;
            }
        }
        v[0] = (double)e;
        v[1] = (double)m;
    } else {
        const T *sp = static_cast<const T *>(G.spins);
        for (int64_t i = t0; i < G.N; i += stride)
            if (!G.occ || bit_of(G.occ, i))
#pragma unroll
                for (int k = 0; k < NC; ++k) v[1 + k] = __dadd_rn(v[1 + k], (double)sp[k * G.N + i]);
        for (int64_t b = t0; b < G.NB; b += stride) {
            if (G.present && !bit_of(G.present, b)) continue;
            int i, j;
            bond_ends(G, b, i, j);
            double d = __dmul_rn((double)sp[i], (double)sp[j]);
#pragma unroll
            for (int k = 1; k < NC; ++k) d = __dadd_rn(d, __dmul_rn((double)sp[k * G.N + i], (double)sp[k * G.N + j]));
            v[0] = __dadd_rn(v[0], d);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double tot = block_sum_f64(v[q]);
        if (threadIdx.x == 0) G.partials[4 * blockIdx.x + q] = tot;
    }
}

// One block: the partials in a fixed order, E = -J sum s_i . s_j,
// m = |M| / N_occ, m^2, m^4; mode 1 adds them to the Neumaier sums and
// advances the sweep counter, mode 2 only records them.
__global__ void __launch_bounds__(1024) graph_accumulate_kernel(const __grid_constant__ GraphDev G, int nblocks,
                                                                int mode)
{
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(v[q], G.partials[4 * b + q]);
    double tot[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) tot[q] = block_sum_f64(v[q]);
    if (threadIdx.x != 0) return;
    DevStats *st = G.st;
    const double E = __dmul_rn(-G.J, tot[0]);
    double m = 0.0;
    if (G.nocc > 0) {
        if (G.nc == 1) {
            m = __ddiv_rn(fabs(tot[1]), (double)G.nocc);
        } else {
            double msq = __dmul_rn(tot[1], tot[1]);
            for (int k = 1; k < G.nc; ++k) msq = __dadd_rn(msq, __dmul_rn(tot[1 + k], tot[1 + k]));
            m = __ddiv_rn(__dsqrt_rn(msq), (double)G.nocc);
        }
    }
    const double m2 = __dmul_rn(m, m);
    const double m4 = __dmul_rn(m2, m2);
    st->last[0] = E;
    st->last[1] = m2;
    st->last[2] = m4;
    st->last[3] = tot[1];
    if (mode != 1) return;
    nsum_add(st->acc_s[0], st->acc_c[0], E);
    nsum_add(st->acc_s[1], st->acc_c[1], __dmul_rn(E, E));
    nsum_add(st->acc_s[2], st->acc_c[2], m2);
    nsum_add(st->acc_s[3], st->acc_c[3], m4);
    nsum_add(st->acc_s[4], st->acc_c[4], __dsqrt_rn(m2));
    st->count += 1;
    st->sweep += 1;
}

__global__ void graph_set_sweep_kernel(DevStats *st, unsigned long long s) { st->sweep = s; }

cudaError_t graph_set_unite_bound(int bound) { return cudaMemcpyToSymbol(c_unite_bound, &bound, sizeof(int)); }

// ------------------------------------------------------------ host side --
static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Kernels of one (model, precision).
struct GraphKernels {
    void (*init)(GraphDev, int, cudaStream_t, unsigned);
    void (*sweep)(const GraphDev &, cudaStream_t, unsigned, unsigned, unsigned, unsigned);
    void (*measure)(const GraphDev &, cudaStream_t, unsigned);
};

template <int NC, typename T>
struct GraphOps {
    static void init(GraphDev G, int random, cudaStream_t s, unsigned nsite_blocks)
    {
        graph_init_kernel<NC, T><<<nsite_blocks, GB_THREADS, 0, s>>>(G, random);
    }
    static void sweep(const GraphDev &G, cudaStream_t s, unsigned nproj, unsigned nbond, unsigned nsite,
                      unsigned nmeas)
    {
        if (NC > 1) graph_proj_kernel<NC, T><<<nproj, GB_THREADS, 0, s>>>(G);
        graph_bond_kernel<NC, T><<<nbond, GB_THREADS, 0, s>>>(G);
        graph_flip_kernel<NC, T><<<nsite, GB_THREADS, 0, s>>>(G);
        graph_measure_kernel<NC, T><<<nmeas, GB_THREADS, 0, s>>>(G);
    }
    static void measure(const GraphDev &G, cudaStream_t s, unsigned nmeas)
    {
        graph_measure_kernel<NC, T><<<nmeas, GB_THREADS, 0, s>>>(G);
    }
};

static GraphKernels kernels_for(int model, int prec)
{
    if (model == PYRO_ISING) return {GraphOps<1, double>::init, GraphOps<1, double>::sweep, GraphOps<1, double>::measure};
    if (model == PYRO_XY) {
        if (prec == PYRO_FP64) return {GraphOps<2, double>::init, GraphOps<2, double>::sweep, GraphOps<2, double>::measure};
        return {GraphOps<2, float>::init, GraphOps<2, float>::sweep, GraphOps<2, float>::measure};
    }
    if (prec == PYRO_FP64) return {GraphOps<3, double>::init, GraphOps<3, double>::sweep, GraphOps<3, double>::measure};
    return {GraphOps<3, float>::init, GraphOps<3, float>::sweep, GraphOps<3, float>::measure};
}

struct GraphEngine {
    GraphDev G{};
    int model = 0, prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void *> owned;
    int32_t *lab_a = nullptr, *lab_b = nullptr, *lab_last = nullptr;
    uint64_t launches = 0;
    double beta = -1.0;
    unsigned nproj = 1, nbond = 1, nsite = 1, nmeas = 1;
    GraphKernels k{};

    cudaError_t alloc(void **p, size_t bytes)
    {
        const cudaError_t e = engine_malloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    }

    void release()
    {
        if (stream) cudaStreamSynchronize(stream);
        for (void *p : owned) cudaFree(p);
        owned.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }

    size_t spin_elem() const { return model == PYRO_ISING ? 1 : (prec == PYRO_FP64 ? 8 : 4); }

    cudaError_t setup(const pyro_graph_config &c, int64_t N, int64_t NB, const std::vector<uint32_t> &present,
                      const std::vector<uint32_t> &occ, int64_t nocc, std::string &err)
    {
        model = c.model;
        prec = model == PYRO_ISING ? PYRO_FP64 : c.precision;
        k = kernels_for(model, prec);
        cudaError_t e;
        if (c.stream) {
            stream = static_cast<cudaStream_t>(c.stream);
        } else {
            e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return err = "stream creation", e;
            own_stream = true;
        }
        G.N = N;
        G.NB = NB;
        G.nocc = nocc;
        G.L = c.sc_L;
        G.nc = model;
        G.seed = c.seed;
        G.J = c.J;
        const int64_t nchunk = std::max(cdiv(NB, 16), cdiv(N, 128));
        nbond = (unsigned)std::max<int64_t>(1, cdiv(nchunk, GB_THREADS));
        nsite = (unsigned)cdiv(N, GB_THREADS);
        nproj = (unsigned)std::min<int64_t>(cdiv(N, GB_THREADS), 152 * 8);
        nmeas = (unsigned)std::min<int64_t>(cdiv(std::max(N, NB), GB_THREADS), 152 * 8);
        struct {
            void **p;
            size_t bytes;
        } al[] = {{&G.spins, (size_t)N * model * spin_elem()},
                  {(void **)&lab_a, (size_t)N * 4},
                  {(void **)&lab_b, (size_t)N * 4},
                  {(void **)&G.fb, (size_t)cdiv(N, 128) * 16},
                  {&G.proj, model == PYRO_ISING ? 0 : (size_t)N * spin_elem()},
                  {(void **)&G.axis, 3 * sizeof(double)},
                  {(void **)&G.partials, (size_t)nmeas * 4 * sizeof(double)},
                  {(void **)&G.st, sizeof(DevStats)},
                  {(void **)&G.bi, c.sc_L ? 0 : (size_t)NB * 4},
                  {(void **)&G.bj, c.sc_L ? 0 : (size_t)NB * 4},
                  {(void **)&G.present, present.size() * 4},
                  {(void **)&G.occ, occ.size() * 4}};
        for (auto &a : al) {
            if (!a.bytes) {
                *a.p = nullptr;
                continue;
            }
            e = alloc(a.p, a.bytes);
            if (e != cudaSuccess) return err = "device allocation failed", e;
        }
        if (!c.sc_L && NB) {
            e = cudaMemcpyAsync(const_cast<int32_t *>(G.bi), c.bond_i, (size_t)NB * 4, cudaMemcpyHostToDevice, stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(const_cast<int32_t *>(G.bj), c.bond_j, (size_t)NB * 4, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return err = "bond list copy", e;
        }
        if (!present.empty()) {
            e = cudaMemcpyAsync(const_cast<uint32_t *>(G.present), present.data(), present.size() * 4,
                                cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return err = "bond mask copy", e;
        }
        if (!occ.empty()) {
            e = cudaMemcpyAsync(const_cast<uint32_t *>(G.occ), occ.data(), occ.size() * 4, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return err = "site mask copy", e;
        }
        e = cudaMemsetAsync(G.st, 0, sizeof(DevStats), stream);
        if (e != cudaSuccess) return err = "stats reset", e;
        G.lab = lab_a;
        G.lab_next = lab_b;
        lab_last = lab_b;
        k.init(G, c.start == PYRO_START_RANDOM, stream, nsite);
        ++launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return err = "init launch", e;
        // the host-side copies above read pageable host memory that the
        // caller may free on return
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return err = "set-up", e;
        return cudaSuccess;
    }

    cudaError_t set_beta(double b)
    {
        if (b == beta) return cudaSuccess;
        beta = b;
        G.thr = ising_threshold(b, G.J);
        G.K2 = 2.0 * b * G.J;
        return cudaSuccess;
    }

    cudaError_t sweeps(int64_t n)
    {
        for (int64_t s = 0; s < n; ++s) {
            k.sweep(G, stream, nproj, nbond, nsite, nmeas);
            graph_accumulate_kernel<<<1, 1024, 0, stream>>>(G, (int)nmeas, 1);
            launches += model == PYRO_ISING ? 4 : 5;
            lab_last = G.lab;
            std::swap(G.lab, G.lab_next);
        }
        return cudaGetLastError();
    }

    cudaError_t measure()
    {
        k.measure(G, stream, nmeas);
        graph_accumulate_kernel<<<1, 1024, 0, stream>>>(G, (int)nmeas, 2);
        launches += 2;
        return cudaGetLastError();
    }

    int read_status(std::string &err)
    {
        int st = 0;
        cudaError_t e = cudaMemcpyAsync(&st, &G.st->status, sizeof(int), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            err = std::string("device status read: ") + cudaGetErrorString(e);
            return -1;
        }
        if (st) cudaMemsetAsync(&G.st->status, 0, sizeof(int), stream);
        return st;
    }
};

}  // namespace pyro

// ------------------------------------------------------------------ C ABI --
struct pyro_graph_ctx {
    pyro::GraphEngine g;
};

namespace pyro {

void set_error(const std::string &msg);

static int gfail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

#define GRAPH_CUDA(call, what)                                                                     \
    do {                                                                                           \
        const cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return gfail(PYRO_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static int gfinish(GraphEngine &g)
{
    std::string err;
    const int st = g.read_status(err);
    if (st < 0) return gfail(PYRO_E_CUDA, err);
    if (st & ST_NOCONVERGE) return gfail(PYRO_E_NOCONVERGE, "union-find exceeded its iteration bound");
    return PYRO_OK;
}

// Bond list of a neighbour table; -1 on a bad table (see pyro.h).
static int64_t bonds_from_table(int64_t N, int z, const int32_t *nbr, int32_t *bi, int32_t *bj, std::string &why)
{
    int64_t E = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < z; ++k) {
            const int32_t j = nbr[i * z + k];
            if (j < 0) continue;
            if (j >= N || j == i) {
                why = "neighbour table entry out of range or naming its own row (site " + std::to_string(i) + ")";
                return -1;
            }
            if (i < j) {
                // j must appear in i's row as often as i appears in j's row
                int a = 0, b = 0;
                for (int q = 0; q < z; ++q) {
                    a += nbr[i * z + q] == j;
                    b += nbr[(int64_t)j * z + q] == i;
                }
                if (a != b) {
                    why = "neighbour table is not symmetric (sites " + std::to_string(i) + ", " + std::to_string(j) + ")";
                    return -1;
                }
                if (bi) {
                    bi[E] = (int32_t)i;
                    bj[E] = j;
                }
                ++E;
            } else {
                int a = 0, b = 0;
                for (int q = 0; q < z; ++q) {
                    a += nbr[i * z + q] == j;
                    b += nbr[(int64_t)j * z + q] == i;
                }
                if (a != b) {
                    why = "neighbour table is not symmetric (sites " + std::to_string(j) + ", " + std::to_string(i) + ")";
                    return -1;
                }
            }
        }
    return E;
}

}  // namespace pyro

using namespace pyro;

extern "C" {

int64_t pyro_graph_bonds_from_table(int64_t N, int z, const int32_t *nbr, int32_t *bond_i, int32_t *bond_j)
{
    if (N < 1 || N > INT32_MAX || z < 0 || (z > 0 && !nbr) || ((bond_i == nullptr) != (bond_j == nullptr)))
        return gfail(PYRO_E_INVAL, "bad argument");
    std::string why;
    const int64_t E = bonds_from_table(N, z, nbr, bond_i, bond_j, why);
    if (E < 0) return gfail(PYRO_E_INVAL, why);
    return E;
}

int pyro_graph_init(pyro_graph *out, const pyro_graph_config *c)
{
    if (!out || !c) return gfail(PYRO_E_INVAL, "NULL argument");
    *out = nullptr;
    if (c->model < PYRO_ISING || c->model > PYRO_HEIS) return gfail(PYRO_E_INVAL, "model must be 1, 2 or 3");
    if (c->model != PYRO_ISING && c->precision != PYRO_FP32 && c->precision != PYRO_FP64)
        return gfail(PYRO_E_INVAL, "precision must be PYRO_FP32 or PYRO_FP64");
    if (c->start != PYRO_START_UP && c->start != PYRO_START_RANDOM)
        return gfail(PYRO_E_INVAL, "start must be PYRO_START_UP or PYRO_START_RANDOM");
    if (!(c->J > 0.0) || !std::isfinite(c->J)) return gfail(PYRO_E_INVAL, "J must be positive and finite");
    int64_t N, NB;
    if (c->sc_L) {
        if (c->sc_L < 2 || c->sc_L > 1290) return gfail(PYRO_E_INVAL, "sc_L must be in [2, 1290]");
        if (c->bond_i || c->bond_j) return gfail(PYRO_E_INVAL, "a simple-cubic lattice takes no bond list");
        N = (int64_t)c->sc_L * c->sc_L * c->sc_L;
        NB = 3 * N;
    } else {
        N = c->nsites;
        NB = c->nbonds;
        if (N < 1 || N > INT32_MAX) return gfail(PYRO_E_INVAL, "nsites must be in [1, 2^31)");
        if (NB < 0 || NB >= ((int64_t)1 << 35)) return gfail(PYRO_E_INVAL, "nbonds must be in [0, 2^35)");
        if (NB && (!c->bond_i || !c->bond_j)) return gfail(PYRO_E_INVAL, "NULL bond list");
        for (int64_t e = 0; e < NB; ++e) {
            const int64_t i = c->bond_i[e], j = c->bond_j[e];
            if (i < 0 || i >= N || j < 0 || j >= N) return gfail(PYRO_E_INVAL, "bond " + std::to_string(e) + ": site out of range");
            if (i == j) return gfail(PYRO_E_INVAL, "bond " + std::to_string(e) + ": self-loop");
        }
    }
    // occupied-site and present-bond bit sets (only with a mask)
    std::vector<uint32_t> occ, present;
    int64_t nocc = N;
    if (c->site_mask) {
        occ.assign((size_t)((N + 31) / 32), 0u);
        nocc = 0;
        for (int64_t i = 0; i < N; ++i)
            if (c->site_mask[i]) {
                occ[(size_t)(i >> 5)] |= 1u << (i & 31);
                ++nocc;
            }
    }
    if (c->site_mask || c->bond_mask) {
        present.assign((size_t)((NB + 31) / 32), 0u);
        const int64_t L = c->sc_L;
        for (int64_t e = 0; e < NB; ++e) {
            if (c->bond_mask && !c->bond_mask[e]) continue;
            int64_t i, j;
            if (L) {
                const int64_t s = e / 3, d = e % 3, x = s % L, y = (s / L) % L, z = s / (L * L);
                i = s;
                j = d == 0 ? (x + 1) % L + L * (y + L * z) : d == 1 ? x + L * ((y + 1) % L + L * z)
                                                                    : x + L * (y + L * ((z + 1) % L));
            } else {
                i = c->bond_i[e];
                j = c->bond_j[e];
            }
            if (c->site_mask && (!c->site_mask[i] || !c->site_mask[j])) continue;
            present[(size_t)(e >> 5)] |= 1u << (e & 31);
        }
    }
    pyro_graph_ctx *h = new (std::nothrow) pyro_graph_ctx;
    if (!h) return gfail(PYRO_E_NOMEM, "host allocation failed");
    std::string err;
    const cudaError_t ce = h->g.setup(*c, N, NB, present, occ, nocc, err);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        h->g.release();
        delete h;
        return gfail(ce == cudaErrorMemoryAllocation ? PYRO_E_NOMEM : PYRO_E_CUDA,
                     err + ": " + cudaGetErrorString(ce));
    }
    *out = h;
    return PYRO_OK;
}

int pyro_graph_sweep(pyro_graph g, double beta, int64_t n)
{
    if (!g) return gfail(PYRO_E_INVAL, "NULL handle");
    if (!(beta >= 0.0) || !std::isfinite(beta)) return gfail(PYRO_E_INVAL, "beta must be finite and >= 0");
    if (n < 0) return gfail(PYRO_E_INVAL, "n must be >= 0");
    g->g.set_beta(beta);
    GRAPH_CUDA(g->g.sweeps(n), "sweep launch");
    return PYRO_OK;
}

int pyro_graph_measure(pyro_graph g, double *E, double *m2, double *m4)
{
    if (!g) return gfail(PYRO_E_INVAL, "NULL handle");
    GRAPH_CUDA(g->g.measure(), "measure launch");
    double last[4];
    GRAPH_CUDA(cudaMemcpyAsync(last, g->g.G.st->last, sizeof(last), cudaMemcpyDeviceToHost, g->g.stream), "measure copy");
    const int rc = gfinish(g->g);
    if (rc) return rc;
    if (E) *E = last[0];
    if (m2) *m2 = last[1];
    if (m4) *m4 = last[2];
    return PYRO_OK;
}

int pyro_graph_stats(pyro_graph g, pyro_stats_t *s)
{
    if (!g || !s) return gfail(PYRO_E_INVAL, "NULL argument");
    DevStats d;
    GRAPH_CUDA(cudaMemcpyAsync(&d, g->g.G.st, sizeof(d), cudaMemcpyDeviceToHost, g->g.stream), "stats copy");
    const int rc = gfinish(g->g);
    if (rc) return rc;
    s->count = d.count;
    double *dst[5] = {&s->sum_E, &s->sum_E2, &s->sum_m2, &s->sum_m4, &s->sum_absm};
    for (int k = 0; k < 5; ++k) *dst[k] = d.acc_s[k] + d.acc_c[k];
    return PYRO_OK;
}

int pyro_graph_reset_stats(pyro_graph g)
{
    if (!g) return gfail(PYRO_E_INVAL, "NULL handle");
    DevStats *d = g->g.G.st;
    GRAPH_CUDA(cudaMemsetAsync(d->acc_s, 0, sizeof(d->acc_s), g->g.stream), "reset");
    GRAPH_CUDA(cudaMemsetAsync(d->acc_c, 0, sizeof(d->acc_c), g->g.stream), "reset");
    GRAPH_CUDA(cudaMemsetAsync(&d->count, 0, sizeof(d->count), g->g.stream), "reset");
    return PYRO_OK;
}

int pyro_graph_get_spins(pyro_graph g, void *host, size_t bytes)
{
    if (!g || !host) return gfail(PYRO_E_INVAL, "NULL argument");
    GraphEngine &e = g->g;
    const int64_t N = e.G.N;
    if (e.model == PYRO_ISING) {
        if (bytes != (size_t)N) return gfail(PYRO_E_INVAL, "Ising spins need N bytes");
        GRAPH_CUDA(cudaMemcpyAsync(host, e.G.spins, (size_t)N, cudaMemcpyDeviceToHost, e.stream), "spins copy");
        return gfinish(e);
    }
    const int n = e.model;
    if (bytes != (size_t)N * n * sizeof(double)) return gfail(PYRO_E_INVAL, "n-vector spins need 8 n N bytes");
    std::vector<unsigned char> raw((size_t)N * n * e.spin_elem());
    GRAPH_CUDA(cudaMemcpyAsync(raw.data(), e.G.spins, raw.size(), cudaMemcpyDeviceToHost, e.stream), "spins copy");
    const int rc = gfinish(e);
    if (rc) return rc;
    double *o = static_cast<double *>(host);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < n; ++k)
            o[i * n + k] = e.prec == PYRO_FP64 ? reinterpret_cast<const double *>(raw.data())[(size_t)k * N + i]
                                               : (double)reinterpret_cast<const float *>(raw.data())[(size_t)k * N + i];
    return PYRO_OK;
}

int pyro_graph_set_spins(pyro_graph g, const void *host, size_t bytes)
{
    if (!g || !host) return gfail(PYRO_E_INVAL, "NULL argument");
    GraphEngine &e = g->g;
    const int64_t N = e.G.N;
    if (e.model == PYRO_ISING) {
        if (bytes != (size_t)N) return gfail(PYRO_E_INVAL, "Ising spins need N bytes");
        const int8_t *s = static_cast<const int8_t *>(host);
        unsigned bad = 0;  // branch-free, so that the check vectorises
        for (int64_t i = 0; i < N; ++i) bad |= (unsigned)((uint8_t)(s[i] + 1) & 0xFDu);  // 0 for -1 and +1 only
        if (bad) return gfail(PYRO_E_INVAL, "Ising spins must be +1 or -1");
        GRAPH_CUDA(cudaMemcpyAsync(e.G.spins, host, (size_t)N, cudaMemcpyHostToDevice, e.stream), "spins copy");
        GRAPH_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
        return PYRO_OK;
    }
    const int n = e.model;
    if (bytes != (size_t)N * n * sizeof(double)) return gfail(PYRO_E_INVAL, "n-vector spins need 8 n N bytes");
    const double *s = static_cast<const double *>(host);
    std::vector<unsigned char> raw((size_t)N * n * e.spin_elem());
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < n; ++k) {
            if (e.prec == PYRO_FP64) reinterpret_cast<double *>(raw.data())[(size_t)k * N + i] = s[i * n + k];
            else reinterpret_cast<float *>(raw.data())[(size_t)k * N + i] = (float)s[i * n + k];
        }
    GRAPH_CUDA(cudaMemcpyAsync(e.G.spins, raw.data(), raw.size(), cudaMemcpyHostToDevice, e.stream), "spins copy");
    GRAPH_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
    return PYRO_OK;
}

int pyro_graph_get_labels(pyro_graph g, int32_t *host, int64_t n)
{
    if (!g || !host) return gfail(PYRO_E_INVAL, "NULL argument");
    if (n != g->g.G.N) return gfail(PYRO_E_INVAL, "labels need N entries");
    GRAPH_CUDA(cudaMemcpyAsync(host, g->g.lab_last, (size_t)n * 4, cudaMemcpyDeviceToHost, g->g.stream), "labels copy");
    return gfinish(g->g);
}

int pyro_graph_set_sweep(pyro_graph g, uint64_t sweep)
{
    if (!g) return gfail(PYRO_E_INVAL, "NULL handle");
    graph_set_sweep_kernel<<<1, 1, 0, g->g.stream>>>(g->g.G.st, sweep);
    GRAPH_CUDA(cudaGetLastError(), "set sweep");
    return PYRO_OK;
}

uint64_t pyro_graph_get_sweep(pyro_graph g)
{
    if (!g) return 0;
    unsigned long long s = 0;
    if (cudaMemcpyAsync(&s, &g->g.G.st->sweep, sizeof(s), cudaMemcpyDeviceToHost, g->g.stream) != cudaSuccess) return 0;
    cudaStreamSynchronize(g->g.stream);
    return s;
}

int64_t pyro_graph_num_sites(pyro_graph g) { return g ? g->g.G.N : 0; }
int64_t pyro_graph_num_bonds(pyro_graph g) { return g ? g->g.G.NB : 0; }

int pyro_graph_sync(pyro_graph g)
{
    if (!g) return gfail(PYRO_E_INVAL, "NULL handle");
    return gfinish(g->g);
}

void *pyro_graph_get_stream(pyro_graph g) { return g ? static_cast<void *>(g->g.stream) : nullptr; }
uint64_t pyro_graph_launch_count(pyro_graph g) { return g ? g->g.launches : 0; }

void pyro_graph_destroy(pyro_graph g)
{
    if (!g) return;
    g->g.release();
    delete g;
}

}  // extern "C"
