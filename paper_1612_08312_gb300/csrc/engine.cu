// engine.cu -- host side of a set of lattices updated together: device
// memory, the replica table, the launch sequence of a sweep, CUDA graphs of
// multi-sweep chunks, and the per-replica measurement / accumulation kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "engine.h"

namespace pyro {

// ising.cu
size_t ising_local_smem(const TileShape &t);
void launch_labels(const Batch &B, int64_t ntiles, cudaStream_t s);
cudaError_t ising_prepare(const TileShape &t);
void ising_launch_init(const Batch &B, int64_t nblocks, int random, cudaStream_t s);
void ising_launch_phase(int p, const Batch &B, int64_t ntiles, cudaStream_t s);
void ising_launch_measure(const Batch &B, int64_t ntiles, cudaStream_t s);
// vector.cu
size_t vec_local_smem(const TileShape &t, int prec);
cudaError_t vec_prepare(int model, int prec, const TileShape &t);
void vec_launch_init(int model, int prec, const Batch &B, int64_t nblocks, int random, cudaStream_t s);
void vec_launch_phase(int p, int model, int prec, const Batch &B, int64_t ntiles, cudaStream_t s);
void vec_launch_measure(int model, int prec, const Batch &B, int64_t ntiles, cudaStream_t s);

// Per replica (one block each): reduce the per-tile partials of the
// measurement kernel in a fixed order, form E, m = |M|/N, m^2, m^4 (Eq. 1,
// Eq. 2) and, in mode 1, add them to the Neumaier sums, append the trace
// record and advance the sweep counter; mode 2 only records them as the last
// measurement.
// With B.fold groups per replica, a first kernel sums each group of a
// replica's tile partials (a contiguous range, fixed order) on its own
// block, so that the accumulation reads B.fold values per replica instead of
// one per tile; one block reading tens of thousands of partials, in FP64 for
// the n-vector models, was the accumulation's whole cost.
template <bool ISING>
__global__ void __launch_bounds__(256) fold_kernel(const __grid_constant__ Batch B)
{
    const int r = blockIdx.x / B.fold, k = blockIdx.x - r * B.fold;
    const int64_t b0 = B.tile_begin[r], n = B.tile_begin[r + 1] - b0;
    const int64_t lo = b0 + n * k / B.fold, hi = b0 + n * (k + 1) / B.fold;
    const int t = threadIdx.x;
    if (ISING) {
        __shared__ unsigned long long su[2][256];
        unsigned long long a = 0, d = 0;
        for (int64_t b = lo + t; b < hi; b += blockDim.x) {
            const unsigned long long *p = reinterpret_cast<const unsigned long long *>(B.partials + 4 * b);
            a += p[0];
            d += p[1];
        }
        su[0][t] = a;
        su[1][t] = d;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (t < o) {
                su[0][t] += su[0][t + o];
                su[1][t] += su[1][t + o];
            }
            __syncthreads();
        }
        if (t == 0) {
            unsigned long long *o = reinterpret_cast<unsigned long long *>(B.folded + 4 * (int64_t)blockIdx.x);
            o[0] = su[0][0];
            o[1] = su[1][0];
        }
    } else {
        __shared__ double sv[4][256];
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t b = lo + t; b < hi; b += blockDim.x)
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(v[q], B.partials[4 * b + q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) sv[q][t] = v[q];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (t < o)
#pragma unroll
                for (int q = 0; q < 4; ++q) sv[q][t] = __dadd_rn(sv[q][t], sv[q][t + o]);
            __syncthreads();
        }
        if (t == 0)
#pragma unroll
            for (int q = 0; q < 4; ++q) B.folded[4 * (int64_t)blockIdx.x + q] = sv[q][0];
    }
}

template <bool ISING>
__global__ void __launch_bounds__(1024) accumulate_kernel(const __grid_constant__ Batch B, int mode, int nc)
{
    const int r = blockIdx.x;
    const Rep &R = B.reps[r];
    DevStats *st = R.st;
    // the replica's tile partials, or its folded groups
    const double *src = B.fold ? B.folded : B.partials;
    const int64_t b0 = B.fold ? (int64_t)r * B.fold : B.tile_begin[r];
    const int64_t b1 = B.fold ? (int64_t)(r + 1) * B.fold : B.tile_begin[r + 1];
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    if (ISING) {
        __shared__ unsigned long long su[2][1024];
        unsigned long long a = 0, d = 0;
        for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
            const unsigned long long *p = reinterpret_cast<const unsigned long long *>(src + 4 * b);
            a += p[0];
            d += p[1];
        }
        su[0][threadIdx.x] = a;
        su[1][threadIdx.x] = d;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                su[0][threadIdx.x] += su[0][threadIdx.x + o];
                su[1][threadIdx.x] += su[1][threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x != 0) return;
        const long long anti = (long long)su[0][0];
        const long long M = R.N - 2 * (long long)su[1][0];
        tot[0] = (double)(3 * R.N - 2 * anti);  // sum over bonds of s_i s_j
        tot[1] = (double)M;
    } else {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x)
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = __dadd_rn(v[q], src[4 * b + q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) tot[q] = block_sum_f64(v[q]);
        if (threadIdx.x != 0) return;
    }
    const double E = __dmul_rn(-R.J, tot[0]);
    double m;
    if (ISING) {
        m = __ddiv_rn(fabs(tot[1]), (double)R.N);
    } else {
        double msq = __dmul_rn(tot[1], tot[1]);
        for (int k = 1; k < nc; ++k) msq = __dadd_rn(msq, __dmul_rn(tot[1 + k], tot[1 + k]));
        m = __ddiv_rn(__dsqrt_rn(msq), (double)R.N);
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
    if (R.trace && R.trace_cap > 0) {
        double *rec = R.trace + 4 * (int64_t)(st->count % (unsigned long long)R.trace_cap);
        rec[0] = E;
        rec[1] = m2;
        rec[2] = m4;
        rec[3] = tot[1];
    }
    st->count += 1;
    st->sweep += 1;
    st->last_epoch = st->epoch;
    st->epoch += 1;
}

__global__ void set_params_kernel(Rep *reps, int r, uint64_t thr, double K2)
{
    reps[r].thr = thr;
    reps[r].K2 = K2;
}

__global__ void set_trace_kernel(Rep *reps, int r, double *trace, int64_t cap)
{
    reps[r].trace = trace;
    reps[r].trace_cap = cap;
}

__global__ void set_sweep_kernel(const __grid_constant__ Batch B, unsigned long long sweep)
{
    if ((int)threadIdx.x < B.R) B.reps[threadIdx.x].st->sweep = sweep;
}

__global__ void reset_epoch_kernel(const __grid_constant__ Batch B)
{
    if ((int)threadIdx.x < B.R) {
        B.reps[threadIdx.x].st->epoch = 0;
        B.reps[threadIdx.x].st->last_epoch = 0xFFFFFFFFull;
    }
}

// Host launcher of the accumulation kernel for callers outside this file.
void launch_accumulate(const Batch &B, bool ising, int mode, int nc, cudaStream_t s)
{
    if (ising) accumulate_kernel<true><<<B.R, 1024, 0, s>>>(B, mode, nc);
    else accumulate_kernel<false><<<B.R, 1024, 0, s>>>(B, mode, nc);
}

// ------------------------------------------------------------------ host --
int g_fail_allocs = 0;
uint64_t g_epoch_start = 0;

cudaError_t engine_malloc(void **p, size_t bytes)
{
    if (g_fail_allocs > 0) {
        --g_fail_allocs;
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

uint64_t ising_threshold(double beta, double J)
{
    if (!(beta > 0.0)) return 0;
    const double p = -expm1(-2.0 * beta * J);
    if (!(p > 0.0)) return 0;
    const double tq = floor(p * 4294967296.0);
    return tq >= 4294967296.0 ? (1ull << 32) : (uint64_t)tq;
}

// Largest power of two that divides L and is at most cap.
static int pow2_divisor_at_most(int L, int cap)
{
    int d = 1;
    while (2 * d <= cap && L % (2 * d) == 0) d *= 2;
    return d;
}

static int log2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

TileShape default_tile(const int *Ls, int R, int model)
{
    int g = Ls[0];
    for (int r = 1; r < R; ++r) {
        int a = g, b = Ls[r];
        while (b) {
            const int t = a % b;
            a = b;
            b = t;
        }
        g = a;
    }
    if (model == PYRO_ISING)  // 8 x 8 x 4 (8 x 8 x 8 is within 1-2 % at L = 256; the autotuner picks per lattice)
        return TileShape{pow2_divisor_at_most(g, 8), pow2_divisor_at_most(g, 8), pow2_divisor_at_most(g, 4)};
    return TileShape{pow2_divisor_at_most(g, 8), pow2_divisor_at_most(g, 4), pow2_divisor_at_most(g, 4)};
}

size_t local_smem(int model, int prec, const TileShape &t)
{
    return model == PYRO_ISING ? ising_local_smem(t) : vec_local_smem(t, prec);
}

std::string check_tile(const int *Ls, int R, int model, int prec, const TileShape &t)
{
    if (!is_pow2(t.TX) || !is_pow2(t.TY) || !is_pow2(t.TZ)) return "tile edges must be powers of two";
    for (int r = 0; r < R; ++r)
        if (Ls[r] % t.TX || Ls[r] % t.TY || Ls[r] % t.TZ) return "tile edges must divide every L";
    const int nt = t.TX * t.TY * t.TZ;
    if (nt > 512) return "tile has too many cells (at most 512)";
    if (local_smem(model, prec, t) > 200 * 1024) return "tile needs too much shared memory";
    return "";
}

static size_t spin_bytes_of(int model, int prec, int64_t N)
{
    if (model == PYRO_ISING) return (size_t)(N / 16) * sizeof(uint16_t);
    return (size_t)N * model * (prec == PYRO_FP64 ? 8 : 4);
}

size_t Engine::spin_bytes(int r) const { return spin_bytes_of(model, prec, reps[r].N); }

static size_t ws_align(size_t x) { return (x + 255) & ~(size_t)255; }

// The replicas' statistics records (contiguous); per replica: spins,
// links, tile-local labels, flip words, face masks, canonical labels; then
// the tiles' partial sums and the replica table.
size_t workspace_bytes(int R, const int *Ls, int model, int prec, const TileShape &t)
{
    size_t total = ws_align((size_t)R * sizeof(DevStats));
    int64_t ntiles = 0;
    const int nt = t.TX * t.TY * t.TZ;
    for (int r = 0; r < R; ++r) {
        const int64_t ncells = (int64_t)Ls[r] * Ls[r] * Ls[r], N = 16 * ncells;
        total += ws_align(spin_bytes_of(model, prec, N)) + ws_align((size_t)N * sizeof(unsigned long long)) +
                 ws_align((size_t)N * sizeof(uint16_t)) + ws_align((size_t)ncells * sizeof(uint16_t)) +
                 ws_align((size_t)ncells * sizeof(uint32_t)) + ws_align((size_t)N * sizeof(int32_t));
        ntiles += ncells / nt;
    }
    return total + ws_align((size_t)(ntiles + (int64_t)R * FOLD_GROUPS) * 4 * sizeof(double)) +
           ws_align((size_t)R * sizeof(Rep));
}

// One device array: carved from the caller's workspace when there is one,
// else allocated (and freed by release()).
cudaError_t Engine::alloc(void **p, size_t bytes)
{
    if (ws) {
        const size_t need = ws_align(bytes);
        if (ws_used + need > ws_bytes) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        *p = ws + ws_used;
        ws_used += need;
        return cudaSuccess;
    }
    const cudaError_t e = engine_malloc(p, bytes);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
}

cudaError_t Engine::setup(int R_, const int *Ls, const double *betas, int model_, int prec_, int start_, double J,
                          const uint64_t *seeds, cudaStream_t user_stream, const TileShape &t, std::string &err,
                          void *workspace, size_t workspace_bytes_)
{
    ws = static_cast<unsigned char *>(workspace);
    ws_bytes = workspace ? workspace_bytes_ : 0;
    ws_used = 0;
    R = R_;
    model = model_;
    prec = model_ == PYRO_ISING ? PYRO_FP64 : prec_;
    start = start_;
    tile = t;
    cudaError_t e = cudaSuccess;
    if (user_stream) {
        stream = user_stream;
        own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            err = "stream create";
            return e;
        }
        own_stream = true;
    }
    std::memset(&B, 0, sizeof(B));
    B.R = R;
    B.TX = t.TX;
    B.TY = t.TY;
    B.TZ = t.TZ;
    B.lTX = log2i(t.TX);
    B.lTY = log2i(t.TY);
    B.lTZ = log2i(t.TZ);
    reps.assign(R, Rep{});
    epoch = g_epoch_start;
    ntiles = 0;
    nblocks = 0;
    const int nt = t.TX * t.TY * t.TZ;
    // every replica's statistics in one block, so that they can be read in
    // one copy
    DevStats *stats = nullptr;
    e = alloc((void **)&stats, (size_t)R * sizeof(DevStats));
    if (e != cudaSuccess) {
        err = ws ? "workspace too small" : "device allocation failed";
        return e;
    }
    for (int r = 0; r < R; ++r) {
        Rep &p = reps[r];
        p.L = Ls[r];
        p.ncells = (int64_t)Ls[r] * Ls[r] * Ls[r];
        p.N = 16 * p.ncells;
        p.ntx = Ls[r] / t.TX;
        p.nty = Ls[r] / t.TY;
        p.seed = seeds[r];
        p.J = J;
        p.thr = ising_threshold(betas ? betas[r] : 0.0, J);
        p.K2 = 2.0 * (betas ? betas[r] : 0.0) * J;
        beta.push_back(betas ? betas[r] : 0.0);
        B.tile_begin[r] = ntiles;
        B.block_begin[r] = nblocks;
        ntiles += p.ncells / nt;
        nblocks += (p.ncells + CELL_BLOCK - 1) / CELL_BLOCK;
        struct {
            void **ptr;
            size_t bytes;
        } al[] = {{&p.spins, spin_bytes_of(model, prec, p.N)},
                  {(void **)&p.P, (size_t)p.N * sizeof(unsigned long long)},
                  {(void **)&p.L16, (size_t)p.N * sizeof(uint16_t)},
                  {(void **)&p.F, (size_t)p.ncells * sizeof(uint16_t)},
                  {(void **)&p.dmask, (size_t)p.ncells * sizeof(uint32_t)},
                  {(void **)&p.labels, ws ? (size_t)p.N * sizeof(int32_t) : 0}};
        p.st = stats + r;
        for (auto &a : al) {
            if (!a.bytes) continue;  // canonical labels: allocated on first use, unless in a workspace
            e = alloc(a.ptr, a.bytes);
            if (e != cudaSuccess) {
                err = ws ? "workspace too small" : "device allocation failed";
                return e;
            }
        }
        e = cudaMemsetAsync(p.st, 0, sizeof(DevStats), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(p.P, 0xFF, (size_t)p.N * sizeof(unsigned long long), stream);
        if (e == cudaSuccess && g_epoch_start) {
            hst_epoch = g_epoch_start;
            e = cudaMemcpyAsync(&p.st->epoch, &hst_epoch, sizeof(hst_epoch), cudaMemcpyHostToDevice, stream);
        }
        if (e != cudaSuccess) return e;
    }
    B.tile_begin[R] = ntiles;
    B.block_begin[R] = nblocks;
    // lattices of many tiles first fold their partials (see fold_kernel)
    int64_t max_tiles = 0;
    for (int r = 0; r < R; ++r) max_tiles = std::max(max_tiles, B.tile_begin[r + 1] - B.tile_begin[r]);
    B.fold = max_tiles >= FOLD_MIN_TILES ? FOLD_GROUPS : 0;
    e = alloc((void **)&B.partials, (size_t)(ntiles + (int64_t)R * FOLD_GROUPS) * 4 * sizeof(double));
    B.folded = B.partials ? B.partials + 4 * ntiles : nullptr;
    if (e == cudaSuccess) e = alloc((void **)&d_reps, (size_t)R * sizeof(Rep));
    if (e != cudaSuccess) {
        err = ws ? "workspace too small" : "device allocation failed";
        return e;
    }
    B.reps = d_reps;
    e = cudaMemcpyAsync(d_reps, reps.data(), (size_t)R * sizeof(Rep), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    e = model == PYRO_ISING ? ising_prepare(tile) : vec_prepare(model, prec, tile);
    if (e != cudaSuccess) {
        err = "kernel attributes";
        return e;
    }
    if (model == PYRO_ISING) ising_launch_init(B, nblocks, start == PYRO_START_RANDOM, stream);
    else vec_launch_init(model, prec, B, nblocks, start == PYRO_START_RANDOM, stream);
    launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) err = "initial state";
    return e;
}

void Engine::release()
{
    if (stream) cudaStreamSynchronize(stream);
    for (auto &g : graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    graphs.clear();
    for (void *p : owned) cudaFree(p);
    owned.clear();
    for (auto &r : reps)
        if (r.trace) cudaFree(r.trace);
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
}

cudaError_t Engine::set_beta(int r, double b)
{
    if (beta[r] == b) return cudaSuccess;
    beta[r] = b;
    reps[r].thr = ising_threshold(b, reps[r].J);
    reps[r].K2 = 2.0 * b * reps[r].J;
    set_params_kernel<<<1, 1, 0, stream>>>(d_reps, r, reps[r].thr, reps[r].K2);
    launches += 1;
    return cudaGetLastError();
}

// Phase p of a sweep: 0 tile-local labelling (with bond activation),
// 1 crossing unions, 2 flip, 3 measurement, 4 accumulation (mode as in
// accumulate_kernel).
void Engine::enqueue_phase(int p, int mode)
{
    if (p < 3) {
        if (model == PYRO_ISING) ising_launch_phase(p, B, ntiles, stream);
        else vec_launch_phase(p, model, prec, B, ntiles, stream);
    } else if (p == 3) {
        if (model == PYRO_ISING) ising_launch_measure(B, ntiles, stream);
        else vec_launch_measure(model, prec, B, ntiles, stream);
    } else {
        if (B.fold) {
            if (model == PYRO_ISING) fold_kernel<true><<<R * B.fold, 256, 0, stream>>>(B);
            else fold_kernel<false><<<R * B.fold, 256, 0, stream>>>(B);
        }
        if (model == PYRO_ISING) accumulate_kernel<true><<<R, 1024, 0, stream>>>(B, mode, 1);
        else accumulate_kernel<false><<<R, 1024, 0, stream>>>(B, mode, model);
    }
}

void Engine::enqueue_sweeps(int n)
{
    for (int s = 0; s < n; ++s)
        for (int p = 0; p < NPHASE; ++p) enqueue_phase(p, 1);
}

void Engine::enqueue_measure(int mode)
{
    enqueue_phase(3, mode);
    enqueue_phase(4, mode);
}

// Crossing-cluster links are stamped with a per-sweep epoch (32 bits).
// Before the epoch could wrap, every link array is reset to "no link" and
// the epochs restart at 0.
cudaError_t Engine::guard_epoch(int n)
{
    if (epoch + (uint64_t)n < 0xFFFFFFF0ull) return cudaSuccess;
    for (auto &r : reps) {
        const cudaError_t e = cudaMemsetAsync(r.P, 0xFF, (size_t)r.N * sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return e;
    }
    reset_epoch_kernel<<<1, MAX_REPS, 0, stream>>>(B);
    launches += 1;
    epoch = 0;
    return cudaGetLastError();
}

cudaError_t Engine::compute_labels()
{
    bool changed = false;
    for (auto &r : reps)
        if (!r.labels) {
            const cudaError_t e = cudaMalloc(&r.labels, (size_t)r.N * sizeof(int32_t));
            if (e != cudaSuccess) return e;
            owned.push_back(r.labels);
            changed = true;
        }
    if (changed) {
        const cudaError_t e = cudaMemcpyAsync(d_reps, reps.data(), (size_t)R * sizeof(Rep), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
    }
    launch_labels(B, ntiles, stream);
    launches += 1;
    return cudaGetLastError();
}

cudaError_t Engine::profile(int n, double *phase_ms)
{
    {
        const cudaError_t e = guard_epoch(n);
        if (e != cudaSuccess) return e;
    }
    epoch += (uint64_t)n;
    cudaEvent_t ev[NPHASE + 1];
    for (auto &x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) return cudaGetLastError();
    double acc[NPHASE] = {};
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < n && e == cudaSuccess; ++s) {
        cudaEventRecord(ev[0], stream);
        for (int p = 0; p < NPHASE; ++p) {
            enqueue_phase(p, 1);
            cudaEventRecord(ev[p + 1], stream);
        }
        launches += launches_per_sweep();
        e = cudaEventSynchronize(ev[NPHASE]);
        for (int p = 0; p < NPHASE && e == cudaSuccess; ++p) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[p], ev[p + 1]);
            acc[p] += ms;
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    sweep += n;
    labels_valid = true;
    for (int p = 0; p < NPHASE; ++p) phase_ms[p] = n > 0 ? acc[p] / n : 0.0;
    return e;
}

// Kernel launches of one sweep: one per phase, the crossing phase is two
// (unions, then the roots' correction bits), and the accumulation two when
// the partials are folded first.
int Engine::launches_per_sweep() const { return NPHASE + 1 + (B.fold ? 1 : 0); }

cudaGraphExec_t Engine::graph_for(int n)
{
    for (auto &g : graphs)
        if (g.n == n) return g.exec;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    enqueue_sweeps(n);
    if (cudaStreamEndCapture(stream, &graph) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    graphs.push_back(GraphEntry{n, exec});
    return exec;
}

cudaError_t Engine::sweeps(int n)
{
    if (n <= 0) return cudaSuccess;
    {
        const cudaError_t e = guard_epoch(n);
        if (e != cudaSuccess) return e;
    }
    epoch += (uint64_t)n;
    if (use_graphs && own_stream) {
        const int chunk = n >= GRAPH_CHUNK ? GRAPH_CHUNK : 1;
        cudaGraphExec_t gk = graph_for(chunk);
        cudaGraphExec_t g1 = chunk == 1 ? gk : graph_for(1);
        if (gk && g1) {
            int left = n;
            while (left >= chunk) {
                const cudaError_t e = cudaGraphLaunch(gk, stream);
                if (e != cudaSuccess) return e;
                left -= chunk;
                launches += (uint64_t)chunk * launches_per_sweep();
            }
            while (left > 0) {
                const cudaError_t e = cudaGraphLaunch(g1, stream);
                if (e != cudaSuccess) return e;
                left -= 1;
                launches += launches_per_sweep();
            }
            sweep += n;
            labels_valid = true;
            return cudaSuccess;
        }
    }
    enqueue_sweeps(n);
    launches += (uint64_t)n * launches_per_sweep();
    sweep += n;
    labels_valid = true;
    return cudaGetLastError();
}

cudaError_t Engine::time_sweeps(int n, double &ms)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    cudaEventRecord(a, stream);
    e = sweeps(n);
    cudaEventRecord(b, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float f = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, a, b);
    ms = n > 0 ? (double)f / n : 0.0;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

cudaError_t Engine::measure()
{
    enqueue_measure(2);
    launches += 2;
    return cudaGetLastError();
}

cudaError_t Engine::set_sweep(uint64_t s)
{
    set_sweep_kernel<<<1, MAX_REPS, 0, stream>>>(B, s);
    launches += 1;
    sweep = s;
    return cudaGetLastError();
}

cudaError_t Engine::set_trace(int r, int64_t cap)
{
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    if (reps[r].trace) cudaFree(reps[r].trace);
    reps[r].trace = nullptr;
    reps[r].trace_cap = 0;
    if (cap > 0) {
        e = cudaMalloc(&reps[r].trace, (size_t)cap * 4 * sizeof(double));
        if (e != cudaSuccess) return e;
        reps[r].trace_cap = cap;
    }
    set_trace_kernel<<<1, 1, 0, stream>>>(d_reps, r, reps[r].trace, reps[r].trace_cap);
    launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e;
}

int Engine::read_status(std::string &err)
{
    // the replicas' records are contiguous: one copy reads every status
    std::vector<DevStats> d((size_t)R);
    cudaError_t e = cudaMemcpyAsync(d.data(), reps[0].st, d.size() * sizeof(DevStats), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return -1;
    }
    int st = 0;
    for (const auto &x : d) st |= x.status;
    return st;
}

}  // namespace pyro
