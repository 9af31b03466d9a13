// api.cu -- the C ABI of libpyro (include/pyro.h): argument checking, error
// reporting and host-side layout conversion around the Engine.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

namespace pyro {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

static int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

static int cuda_fail(cudaError_t e, const std::string &what)
{
    return fail(PYRO_E_CUDA, what + ": " + cudaGetErrorString(e));
}

#define PYRO_CUDA(call, what)                               \
    do {                                                    \
        const cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

static int finish(Engine &e)
{
    std::string err;
    const int st = e.read_status(err);
    if (st < 0) return fail(PYRO_E_CUDA, err);
    if (st & ST_NOCONVERGE) return fail(PYRO_E_NOCONVERGE, "union-find exceeded its iteration bound");
    if (st & ST_TIMEOUT) return fail(PYRO_E_TIMEOUT, "a device wait exceeded its time bound");
    return PYRO_OK;
}

static bool beta_ok(double b) { return b >= 0.0 && std::isfinite(b); }

// Argument checks and the resolved tile of a set of lattices; "" if valid.
static std::string check_args(int R, const int *Ls, const double *betas, int model, int prec, int start, double J,
                              const int tile[3], TileShape &t)
{
    if (R < 1 || R > MAX_REPS) return "number of replicas must be in [1, 64]";
    for (int r = 0; r < R; ++r) {
        if (Ls[r] < 1 || Ls[r] > PYRO_MAX_L) return "L must be in [1, 511]";
        if (betas && !beta_ok(betas[r])) return "beta must be finite and >= 0";
    }
    if (model < PYRO_ISING || model > PYRO_HEIS) return "model must be 1, 2 or 3";
    if (prec != PYRO_FP32 && prec != PYRO_FP64) return "precision must be PYRO_FP32 or PYRO_FP64";
    if (start != PYRO_START_UP && start != PYRO_START_RANDOM) return "start must be PYRO_START_UP or PYRO_START_RANDOM";
    if (!(J > 0.0) || !std::isfinite(J)) return "J must be positive and finite";
    t = default_tile(Ls, R, model);
    if (tile && (tile[0] || tile[1] || tile[2])) t = TileShape{tile[0], tile[1], tile[2]};
    return check_tile(Ls, R, model, prec, t);
}

static int create(Engine &e, int R, const int *Ls, const double *betas, int model, int prec, int start, double J,
                  const uint64_t *seeds, void *stream, const int tile[3], void *workspace = nullptr,
                  size_t workspace_bytes_ = 0)
{
    TileShape t;
    const std::string why = check_args(R, Ls, betas, model, prec, start, J, tile, t);
    if (!why.empty()) return fail(PYRO_E_INVAL, why);
    std::string err;
    if (workspace) {
        if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(PYRO_E_INVAL, "workspace must be 256-byte aligned");
        const size_t need = workspace_bytes(R, Ls, model, model == PYRO_ISING ? PYRO_FP64 : prec, t);
        if (workspace_bytes_ < need)
            return fail(PYRO_E_NOMEM, "workspace too small: " + std::to_string(workspace_bytes_) + " bytes, " +
                                          std::to_string(need) + " needed");
    }
    const cudaError_t ce = e.setup(R, Ls, betas, model, prec, start, J, seeds, static_cast<cudaStream_t>(stream), t, err,
                                   workspace, workspace_bytes_);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        e.release();
        if (ce == cudaErrorMemoryAllocation) return fail(PYRO_E_NOMEM, err + ": " + cudaGetErrorString(ce));
        return cuda_fail(ce, err);
    }
    return PYRO_OK;
}

static size_t vec_elem(const Engine &e) { return e.prec == PYRO_FP64 ? 8 : 4; }

static int get_spins(Engine &e, int r, void *host, size_t bytes)
{
    const int64_t N = e.reps[r].N;
    if (e.model == PYRO_ISING) {
        if (bytes != (size_t)N) return fail(PYRO_E_INVAL, "Ising spins need N bytes");
        std::vector<uint16_t> w((size_t)(N / 16));
        PYRO_CUDA(cudaMemcpyAsync(w.data(), e.reps[r].spins, w.size() * 2, cudaMemcpyDeviceToHost, e.stream), "spins copy");
        PYRO_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
        int8_t *o = static_cast<int8_t *>(host);
        for (int64_t i = 0; i < N; ++i) o[i] = ((w[i >> 4] >> (i & 15)) & 1) ? -1 : 1;
        return PYRO_OK;
    }
    const int n = e.model;
    if (bytes != (size_t)N * n * sizeof(double)) return fail(PYRO_E_INVAL, "n-vector spins need 8 n N bytes");
    std::vector<unsigned char> raw((size_t)N * n * vec_elem(e));
    PYRO_CUDA(cudaMemcpyAsync(raw.data(), e.reps[r].spins, raw.size(), cudaMemcpyDeviceToHost, e.stream), "spins copy");
    PYRO_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
    double *o = static_cast<double *>(host);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < n; ++k)
            o[i * n + k] = e.prec == PYRO_FP64 ? reinterpret_cast<const double *>(raw.data())[(size_t)k * N + i]
                                               : (double)reinterpret_cast<const float *>(raw.data())[(size_t)k * N + i];
    return PYRO_OK;
}

static int stats_of(Engine &e, int r, pyro_stats_t *s)
{
    DevStats d;
    PYRO_CUDA(cudaMemcpyAsync(&d, e.reps[r].st, sizeof(d), cudaMemcpyDeviceToHost, e.stream), "stats copy");
    const int rc = finish(e);
    if (rc) return rc;
    s->count = d.count;
    double *dst[5] = {&s->sum_E, &s->sum_E2, &s->sum_m2, &s->sum_m4, &s->sum_absm};
    for (int k = 0; k < 5; ++k) *dst[k] = d.acc_s[k] + d.acc_c[k];
    return PYRO_OK;
}

static int reset_stats(Engine &e)
{
    for (int r = 0; r < e.R; ++r) {
        DevStats *d = e.reps[r].st;
        PYRO_CUDA(cudaMemsetAsync(d->acc_s, 0, sizeof(d->acc_s), e.stream), "reset");
        PYRO_CUDA(cudaMemsetAsync(d->acc_c, 0, sizeof(d->acc_c), e.stream), "reset");
        PYRO_CUDA(cudaMemsetAsync(&d->count, 0, sizeof(d->count), e.stream), "reset");
    }
    return PYRO_OK;
}

// Every replica's statistics (DevStats records are contiguous): one
// device-to-host copy.
static int stats_all(Engine &e, pyro_stats_t *s)
{
    std::vector<DevStats> d((size_t)e.R);
    PYRO_CUDA(cudaMemcpyAsync(d.data(), e.reps[0].st, d.size() * sizeof(DevStats), cudaMemcpyDeviceToHost, e.stream),
              "stats copy");
    const int rc = finish(e);
    if (rc) return rc;
    for (int r = 0; r < e.R; ++r) {
        s[r].count = d[r].count;
        double *dst[5] = {&s[r].sum_E, &s[r].sum_E2, &s[r].sum_m2, &s[r].sum_m4, &s[r].sum_absm};
        for (int k = 0; k < 5; ++k) *dst[k] = d[r].acc_s[k] + d[r].acc_c[k];
    }
    return PYRO_OK;
}

// Every replica's instantaneous E, m^2, m^4 (out[3 r + 0..2]): one
// measurement launch over all replicas and one device-to-host copy.
static int measure_all(Engine &e, double *out)
{
    PYRO_CUDA(e.measure(), "measure launch");
    std::vector<DevStats> d((size_t)e.R);
    PYRO_CUDA(cudaMemcpyAsync(d.data(), e.reps[0].st, d.size() * sizeof(DevStats), cudaMemcpyDeviceToHost, e.stream),
              "measure copy");
    const int rc = finish(e);
    if (rc) return rc;
    for (int r = 0; r < e.R; ++r)
        for (int k = 0; k < 3; ++k) out[3 * r + k] = d[r].last[k];
    return PYRO_OK;
}

static int measure_of(Engine &e, int r, double *E, double *m2, double *m4)
{
    PYRO_CUDA(e.measure(), "measure launch");
    double last[4];
    PYRO_CUDA(cudaMemcpyAsync(last, e.reps[r].st->last, sizeof(last), cudaMemcpyDeviceToHost, e.stream), "measure copy");
    const int rc = finish(e);
    if (rc) return rc;
    if (E) *E = last[0];
    if (m2) *m2 = last[1];
    if (m4) *m4 = last[2];
    return PYRO_OK;
}

cudaError_t ising_set_unite_bound(int bound);
int noalloc_set_stamp(uint32_t stamp);
cudaError_t vec_set_unite_bound(int bound);
cudaError_t graph_set_unite_bound(int bound);

// ------------------------------------------------------------- autotuner --
// Candidate tiles: powers of two, 64 to 512 cells, each edge dividing L
// (for a set of lattices, their greatest common divisor).
static std::vector<TileShape> tile_candidates(int L, int model)
{
    std::vector<TileShape> out;
    const int edges[] = {2, 4, 8, 16, 32};
    for (int tx : edges)
        for (int ty : edges)
            for (int tz : edges) {
                const int nt = tx * ty * tz;
                if (nt < 64 || nt > 512 || L % tx || L % ty || L % tz || ty > tx) continue;
                if (model != PYRO_ISING && nt > 256) continue;
                out.push_back(TileShape{tx, ty, tz});
            }
    return out;
}

static std::mutex tune_mutex;
static std::map<std::tuple<std::string, std::string, int, int>, std::pair<TileShape, double>> tune_cache;

static std::string device_name()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string n = p.name;
    for (auto &ch : n)
        if (ch == ' ') ch = '_';
    return n;
}

// Optional file cache named by PYRO_AUTOTUNE_CACHE: lines
// "<gpu> <sizes> <model> <precision> <TX> <TY> <TZ> <ms>", sizes the
// lattice's L or a batch's distinct L joined by commas.
static bool file_lookup(const std::string &gpu, const std::string &L, int model, int prec, TileShape &t, double &ms)
{
    const char *path = std::getenv("PYRO_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char name[256];
    int m, p, tx, ty, tz;
    double v;
    bool found = false;
    char sizes[256];
    while (std::fscanf(f, "%255s %255s %d %d %d %d %d %lf", name, sizes, &m, &p, &tx, &ty, &tz, &v) == 8)
        if (gpu == name && L == sizes && m == model && p == prec) {
            t = TileShape{tx, ty, tz};
            ms = v;
            found = true;
        }
    std::fclose(f);
    return found;
}

static void file_store(const std::string &gpu, const std::string &L, int model, int prec, const TileShape &t, double ms)
{
    const char *path = std::getenv("PYRO_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %s %d %d %d %d %d %.6f\n", gpu.c_str(), L.c_str(), model, prec, t.TX, t.TY, t.TZ, ms);
    std::fclose(f);
}

}  // namespace pyro

using namespace pyro;

extern "C" {

const char *pyro_last_error(void) { return g_err.c_str(); }

int pyro_init_ex(pyro_handle *out, const pyro_config *cfg)
{
    if (!out || !cfg) return fail(PYRO_E_INVAL, "NULL argument");
    *out = nullptr;
    pyro_ctx *h = new (std::nothrow) pyro_ctx();
    if (!h) return fail(PYRO_E_NOMEM, "host allocation failed");
    const double beta0 = 0.0;
    const int rc = create(h->e, 1, &cfg->L, &beta0, cfg->model, cfg->precision, cfg->start, cfg->J, &cfg->seed,
                          cfg->stream, cfg->tile, cfg->workspace, cfg->workspace_bytes);
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return PYRO_OK;
}

size_t pyro_workspace_bytes(const pyro_config *cfg)
{
    if (!cfg) {
        set_error("NULL argument");
        return 0;
    }
    const double beta0 = 0.0;
    TileShape t;
    const std::string why =
        check_args(1, &cfg->L, &beta0, cfg->model, cfg->precision, cfg->start, cfg->J, cfg->tile, t);
    if (!why.empty()) {
        set_error(why);
        return 0;
    }
    return workspace_bytes(1, &cfg->L, cfg->model, cfg->model == PYRO_ISING ? PYRO_FP64 : cfg->precision, t);
}

int pyro_init(pyro_handle *out, int L, int model, uint64_t seed)
{
    pyro_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.L = L;
    cfg.model = model;
    cfg.precision = PYRO_FP32;
    cfg.start = PYRO_START_UP;
    cfg.J = 1.0;
    cfg.seed = seed;
    return pyro_init_ex(out, &cfg);
}

int pyro_sweep(pyro_handle h, double beta, int n)
{
    if (!h) return fail(PYRO_E_INVAL, "NULL handle");
    if (!beta_ok(beta)) return fail(PYRO_E_INVAL, "beta must be finite and >= 0");
    if (n < 0) return fail(PYRO_E_INVAL, "n must be >= 0");
    if (n == 0) return PYRO_OK;
    PYRO_CUDA(h->e.set_beta(0, beta), "parameter update");
    PYRO_CUDA(h->e.sweeps(n), "sweep launch");
    return PYRO_OK;
}

int pyro_measure(pyro_handle h, double *E, double *m2, double *m4)
{
    if (!h) return fail(PYRO_E_INVAL, "NULL handle");
    return measure_of(h->e, 0, E, m2, m4);
}

int pyro_stats(pyro_handle h, pyro_stats_t *s)
{
    if (!h || !s) return fail(PYRO_E_INVAL, "NULL argument");
    return stats_of(h->e, 0, s);
}

int pyro_reset_stats(pyro_handle h)
{
    if (!h) return fail(PYRO_E_INVAL, "NULL handle");
    return reset_stats(h->e);
}

size_t pyro_state_bytes(pyro_handle h) { return h ? h->e.spin_bytes(0) : 0; }

int pyro_get_state(pyro_handle h, void *host, size_t bytes)
{
    if (!h || !host) return fail(PYRO_E_INVAL, "NULL argument");
    if (bytes != h->e.spin_bytes(0)) return fail(PYRO_E_INVAL, "state size mismatch");
    PYRO_CUDA(cudaMemcpyAsync(host, h->e.reps[0].spins, bytes, cudaMemcpyDeviceToHost, h->e.stream), "state copy");
    return PYRO_OK;
}

int pyro_set_state(pyro_handle h, const void *host, size_t bytes)
{
    if (!h || !host) return fail(PYRO_E_INVAL, "NULL argument");
    if (bytes != h->e.spin_bytes(0)) return fail(PYRO_E_INVAL, "state size mismatch");
    PYRO_CUDA(cudaMemcpyAsync(h->e.reps[0].spins, host, bytes, cudaMemcpyHostToDevice, h->e.stream), "state copy");
    h->e.labels_valid = false;
    return PYRO_OK;
}

int pyro_get_spins(pyro_handle h, void *host, size_t bytes)
{
    if (!h || !host) return fail(PYRO_E_INVAL, "NULL argument");
    return get_spins(h->e, 0, host, bytes);
}

int pyro_set_spins(pyro_handle h, const void *host, size_t bytes)
{
    if (!h || !host) return fail(PYRO_E_INVAL, "NULL argument");
    Engine &e = h->e;
    const int64_t N = e.reps[0].N;
    if (e.model == PYRO_ISING) {
        if (bytes != (size_t)N) return fail(PYRO_E_INVAL, "Ising spins need N bytes");
        const int8_t *s = static_cast<const int8_t *>(host);
        std::vector<uint16_t> w((size_t)(N / 16), 0);
        for (int64_t i = 0; i < N; ++i) {
            if (s[i] != 1 && s[i] != -1) return fail(PYRO_E_INVAL, "Ising spins must be +1 or -1");
            if (s[i] == -1) w[i >> 4] |= (uint16_t)(1u << (i & 15));
        }
        PYRO_CUDA(cudaMemcpyAsync(e.reps[0].spins, w.data(), w.size() * 2, cudaMemcpyHostToDevice, e.stream), "spins copy");
        PYRO_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
    } else {
        const int n = e.model;
        if (bytes != (size_t)N * n * sizeof(double)) return fail(PYRO_E_INVAL, "n-vector spins need 8 n N bytes");
        const double *s = static_cast<const double *>(host);
        std::vector<unsigned char> raw((size_t)N * n * vec_elem(e));
        for (int64_t i = 0; i < N; ++i)
            for (int k = 0; k < n; ++k) {
                if (e.prec == PYRO_FP64) reinterpret_cast<double *>(raw.data())[(size_t)k * N + i] = s[i * n + k];
                else reinterpret_cast<float *>(raw.data())[(size_t)k * N + i] = (float)s[i * n + k];
            }
        PYRO_CUDA(cudaMemcpyAsync(e.reps[0].spins, raw.data(), raw.size(), cudaMemcpyHostToDevice, e.stream), "spins copy");
        PYRO_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
    }
    e.labels_valid = false;
    return PYRO_OK;
}

int pyro_get_labels(pyro_handle h, int32_t *host, size_t bytes)
{
    if (!h || !host) return fail(PYRO_E_INVAL, "NULL argument");
    if (bytes != (size_t)h->e.reps[0].N * sizeof(int32_t)) return fail(PYRO_E_INVAL, "labels need 4 N bytes");
    if (!h->e.labels_valid) return fail(PYRO_E_STATE, "no sweep since the spins were last set");
    PYRO_CUDA(h->e.compute_labels(), "labels");
    PYRO_CUDA(cudaMemcpyAsync(host, h->e.reps[0].labels, bytes, cudaMemcpyDeviceToHost, h->e.stream), "labels copy");
    return finish(h->e);
}

int pyro_get_sweep(pyro_handle h, uint64_t *sweep)
{
    if (!h || !sweep) return fail(PYRO_E_INVAL, "NULL argument");
    *sweep = h->e.sweep;
    return PYRO_OK;
}

int pyro_set_sweep(pyro_handle h, uint64_t sweep)
{
    if (!h) return fail(PYRO_E_INVAL, "NULL handle");
    PYRO_CUDA(h->e.set_sweep(sweep), "sweep update");
    return PYRO_OK;
}

int pyro_set_trace(pyro_handle h, int64_t capacity)
{
    if (!h || capacity < 0) return fail(PYRO_E_INVAL, "bad argument");
    const cudaError_t e = h->e.set_trace(0, capacity);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(PYRO_E_NOMEM, "trace allocation failed");
    }
    PYRO_CUDA(e, "trace setup");
    return PYRO_OK;
}

int pyro_get_trace(pyro_handle h, double *host, int64_t max_records, int64_t *n)
{
    if (!h || !host || !n || max_records < 0) return fail(PYRO_E_INVAL, "bad argument");
    *n = 0;
    Engine &e = h->e;
    const int64_t cap = e.reps[0].trace_cap;
    if (!cap) return PYRO_OK;
    unsigned long long count = 0;
    PYRO_CUDA(cudaMemcpyAsync(&count, &e.reps[0].st->count, sizeof(count), cudaMemcpyDeviceToHost, e.stream), "count");
    const int rc = finish(e);
    if (rc) return rc;
    const int64_t have = (int64_t)std::min<unsigned long long>(count, (unsigned long long)cap);
    const int64_t take = std::min<int64_t>(have, max_records);
    std::vector<double> all((size_t)cap * 4);
    PYRO_CUDA(cudaMemcpyAsync(all.data(), e.reps[0].trace, all.size() * sizeof(double), cudaMemcpyDeviceToHost, e.stream),
              "trace copy");
    PYRO_CUDA(cudaStreamSynchronize(e.stream), "stream synchronize");
    for (int64_t q = 0; q < take; ++q) {
        const unsigned long long c = count - (unsigned long long)take + (unsigned long long)q;
        std::memcpy(host + 4 * q, all.data() + 4 * (c % (unsigned long long)cap), 4 * sizeof(double));
    }
    *n = take;
    return PYRO_OK;
}

int pyro_sync(pyro_handle h)
{
    if (!h) return fail(PYRO_E_INVAL, "NULL handle");
    return finish(h->e);
}

int64_t pyro_num_sites(pyro_handle h) { return h ? h->e.reps[0].N : 0; }

int pyro_get_tile(pyro_handle h, int tile[3])
{
    if (!h || !tile) return fail(PYRO_E_INVAL, "NULL argument");
    tile[0] = h->e.tile.TX;
    tile[1] = h->e.tile.TY;
    tile[2] = h->e.tile.TZ;
    return PYRO_OK;
}

void *pyro_get_stream(pyro_handle h) { return h ? (void *)h->e.stream : nullptr; }

int pyro_set_graphs(pyro_handle h, int on)
{
    if (!h) return fail(PYRO_E_INVAL, "NULL handle");
    h->e.use_graphs = on != 0;
    return PYRO_OK;
}

}  // extern "C"

namespace pyro {

// Fastest tile for a set of R lattices (sizes Ls, inverse temperatures
// betas): equilibrate them with the default tile, then replay the same
// sweeps from that state with every candidate tile.  The chain does not
// depend on the tile, so every candidate does identical work.
static int autotune_set(int R, const int *Ls, const double *betas, int model, int precision, int nsweeps,
                        int tile_out[3], double *ms_per_sweep)
{
    if (!tile_out || !Ls || !betas) return fail(PYRO_E_INVAL, "NULL argument");
    if (R < 1 || R > MAX_REPS) return fail(PYRO_E_INVAL, "number of replicas must be in [1, 64]");
    int g = 0;
    std::vector<int> sizes;
    for (int r = 0; r < R; ++r) {
        if (Ls[r] < 1 || Ls[r] > PYRO_MAX_L) return fail(PYRO_E_INVAL, "L must be in [1, 511]");
        if (!beta_ok(betas[r])) return fail(PYRO_E_INVAL, "beta must be >= 0");
        int a = g, b = Ls[r];
        while (b) {
            const int t = a % b;
            a = b;
            b = t;
        }
        g = a;
        sizes.push_back(Ls[r]);
    }
    if (model < PYRO_ISING || model > PYRO_HEIS) return fail(PYRO_E_INVAL, "model must be 1, 2 or 3");
    if (precision != PYRO_FP32 && precision != PYRO_FP64) return fail(PYRO_E_INVAL, "bad precision");
    if (nsweeps < 1) return fail(PYRO_E_INVAL, "nsweeps must be >= 1");
    const int prec = model == PYRO_ISING ? PYRO_FP64 : precision;
    std::sort(sizes.begin(), sizes.end());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    std::string skey;
    for (size_t k = 0; k < sizes.size(); ++k) skey += (k ? "," : "") + std::to_string(sizes[k]);
    const std::string gpu = device_name();
    std::lock_guard<std::mutex> lock(tune_mutex);
    const auto key = std::make_tuple(gpu, skey, model, prec);
    TileShape best = default_tile(Ls, R, model);
    double best_ms = -1.0;
    auto it = tune_cache.find(key);
    if (it != tune_cache.end()) {
        best = it->second.first;
        best_ms = it->second.second;
    } else if (!file_lookup(gpu, skey, model, prec, best, best_ms)) {
        std::vector<uint64_t> seeds((size_t)R);
        for (int r = 0; r < R; ++r) seeds[r] = 0x5EEDull + (uint64_t)r * 0x9E3779B97F4A7C15ull;
        const int warm = 60;
        Engine ref;
        std::string err;
        const TileShape t0 = default_tile(Ls, R, model);
        if (ref.setup(R, Ls, betas, model, prec, PYRO_START_RANDOM, 1.0, seeds.data(), nullptr, t0, err) != cudaSuccess ||
            ref.sweeps(warm) != cudaSuccess || cudaStreamSynchronize(ref.stream) != cudaSuccess) {
            cudaGetLastError();
            ref.release();
            return fail(PYRO_E_CUDA, "autotune: reference lattices failed");
        }
        for (const TileShape &t : tile_candidates(g, model)) {
            if (!check_tile(Ls, R, model, prec, t).empty()) continue;
            Engine e;
            if (e.setup(R, Ls, betas, model, prec, PYRO_START_RANDOM, 1.0, seeds.data(), nullptr, t, err) != cudaSuccess) {
                cudaGetLastError();
                e.release();
                continue;
            }
            e.use_graphs = false;
            double ms = 0.0;
            cudaError_t ce = cudaSuccess;
            for (int r = 0; r < R && ce == cudaSuccess; ++r)
                ce = cudaMemcpyAsync(e.reps[r].spins, ref.reps[r].spins, ref.spin_bytes(r), cudaMemcpyDeviceToDevice,
                                     e.stream);
            if (ce == cudaSuccess) ce = e.set_sweep(ref.sweep);
            if (ce == cudaSuccess) ce = e.sweeps(1);
            if (ce == cudaSuccess) ce = e.time_sweeps(nsweeps, ms);
            e.release();
            if (ce != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (best_ms < 0.0 || ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
        ref.release();
        if (best_ms >= 0.0) file_store(gpu, skey, model, prec, best, best_ms);
    }
    tune_cache[key] = std::make_pair(best, best_ms);
    tile_out[0] = best.TX;
    tile_out[1] = best.TY;
    tile_out[2] = best.TZ;
    if (ms_per_sweep) *ms_per_sweep = best_ms;
    return PYRO_OK;
}

}  // namespace pyro

extern "C" {

int pyro_autotune(int L, int model, int precision, double beta, int nsweeps, int tile_out[3], double *ms_per_sweep)
{
    if (!tile_out) return fail(PYRO_E_INVAL, "NULL argument");
    return autotune_set(1, &L, &beta, model, precision, nsweeps, tile_out, ms_per_sweep);
}

int pyro_batch_autotune(int R, const int *L, const double *beta, int model, int precision, int nsweeps, int tile_out[3],
                        double *ms_per_sweep)
{
    return autotune_set(R, L, beta, model, precision, nsweeps, tile_out, ms_per_sweep);
}

int pyro_debug_set(int key, int64_t value)
{
    if (key == PYRO_DEBUG_FAIL_ALLOCS) {
        if (value < 0) return fail(PYRO_E_INVAL, "count must be >= 0");
        g_fail_allocs = (int)value;
        return PYRO_OK;
    }
    if (key == PYRO_DEBUG_NOALLOC_STAMP) {
        if (value < 0 || value > 0xFFFFFFFFll) return fail(PYRO_E_INVAL, "stamp must be a 32-bit value");
        if (noalloc_set_stamp((uint32_t)value)) return fail(PYRO_E_CUDA, "no current device");
        return PYRO_OK;
    }
    if (key == PYRO_DEBUG_EPOCH_START) {
        if (value < 0 || value > 0xFFFFFFFFll) return fail(PYRO_E_INVAL, "stamp must be a 32-bit value");
        g_epoch_start = (uint64_t)value;
        return PYRO_OK;
    }
    if (key == PYRO_DEBUG_UNITE_BOUND) {
        const int b = value <= 0 ? 0 : (value > 4096 ? 4096 : (int)value);
        PYRO_CUDA(ising_set_unite_bound(b), "bound update");
        PYRO_CUDA(vec_set_unite_bound(b), "bound update");
        PYRO_CUDA(graph_set_unite_bound(b), "bound update");
        return PYRO_OK;
    }
    return fail(PYRO_E_INVAL, "unknown debug key");
}

uint64_t pyro_launch_count(pyro_handle h) { return h ? h->e.launches : 0; }

int pyro_profile_phases(pyro_handle h, double beta, int n, double *phase_ms)
{
    if (!h || !phase_ms) return fail(PYRO_E_INVAL, "NULL argument");
    if (!beta_ok(beta)) return fail(PYRO_E_INVAL, "beta must be finite and >= 0");
    if (n < 1) return fail(PYRO_E_INVAL, "n must be >= 1");
    PYRO_CUDA(h->e.set_beta(0, beta), "parameter update");
    PYRO_CUDA(h->e.profile(n, phase_ms), "profiled sweep");
    return finish(h->e);
}

void pyro_destroy(pyro_handle h)
{
    if (!h) return;
    h->e.release();
    delete h;
}

// ------------------------------------------------------------- batches --
int pyro_batch_init(pyro_batch *out, int R, const int *L, const double *beta, int model, int precision, int start,
                    uint64_t seed)
{
    return pyro_batch_init_ex(out, R, L, beta, model, precision, start, seed, nullptr);
}

int pyro_batch_init_ex(pyro_batch *out, int R, const int *L, const double *beta, int model, int precision, int start,
                       uint64_t seed, const int tile[3])
{
    if (!out || !L || !beta) return fail(PYRO_E_INVAL, "NULL argument");
    *out = nullptr;
    if (R < 1 || R > MAX_REPS) return fail(PYRO_E_INVAL, "number of replicas must be in [1, 64]");
    std::vector<uint64_t> seeds((size_t)R);
    for (int r = 0; r < R; ++r) seeds[r] = seed + (uint64_t)r * 0x9E3779B97F4A7C15ull;
    pyro_batch_ctx *b = new (std::nothrow) pyro_batch_ctx();
    if (!b) return fail(PYRO_E_NOMEM, "host allocation failed");
    const int rc = create(b->e, R, L, beta, model, precision, start, 1.0, seeds.data(), nullptr, tile);
    if (rc) {
        delete b;
        return rc;
    }
    *out = b;
    return PYRO_OK;
}

int pyro_batch_sweep(pyro_batch b, int n)
{
    if (!b) return fail(PYRO_E_INVAL, "NULL handle");
    if (n < 0) return fail(PYRO_E_INVAL, "n must be >= 0");
    PYRO_CUDA(b->e.sweeps(n), "sweep launch");
    return PYRO_OK;
}

int pyro_batch_stats(pyro_batch b, int r, pyro_stats_t *s)
{
    if (!b || !s || r < 0 || r >= b->e.R) return fail(PYRO_E_INVAL, "bad argument");
    return stats_of(b->e, r, s);
}

int pyro_batch_stats_all(pyro_batch b, pyro_stats_t *s)
{
    if (!b || !s) return fail(PYRO_E_INVAL, "NULL argument");
    return stats_all(b->e, s);
}

int pyro_batch_measure_all(pyro_batch b, double *out)
{
    if (!b || !out) return fail(PYRO_E_INVAL, "NULL argument");
    return measure_all(b->e, out);
}

int pyro_batch_reset_stats(pyro_batch b)
{
    if (!b) return fail(PYRO_E_INVAL, "NULL handle");
    return reset_stats(b->e);
}

int pyro_batch_measure(pyro_batch b, int r, double *E, double *m2, double *m4)
{
    if (!b || r < 0 || r >= b->e.R) return fail(PYRO_E_INVAL, "bad argument");
    return measure_of(b->e, r, E, m2, m4);
}

int pyro_batch_get_spins(pyro_batch b, int r, void *host, size_t bytes)
{
    if (!b || !host || r < 0 || r >= b->e.R) return fail(PYRO_E_INVAL, "bad argument");
    return get_spins(b->e, r, host, bytes);
}

int pyro_batch_sync(pyro_batch b)
{
    if (!b) return fail(PYRO_E_INVAL, "NULL handle");
    return finish(b->e);
}

int64_t pyro_batch_total_sites(pyro_batch b)
{
    if (!b) return 0;
    int64_t n = 0;
    for (const auto &r : b->e.reps) n += r.N;
    return n;
}

uint64_t pyro_batch_launch_count(pyro_batch b) { return b ? b->e.launches : 0; }

void *pyro_batch_get_stream(pyro_batch b) { return b ? (void *)b->e.stream : nullptr; }

void pyro_batch_destroy(pyro_batch b)
{
    if (!b) return;
    b->e.release();
    delete b;
}

}  // extern "C"
