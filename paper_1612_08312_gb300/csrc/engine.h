// engine.h -- host-side engine of one or more lattices updated together.
#pragma once

#include <string>
#include <vector>

#include "ccl.cuh"

namespace pyro {

// Sweeps captured per CUDA graph for long runs.
constexpr int GRAPH_CHUNK = 32;
// Phases of a sweep: tile-local labelling, crossing unions (two launches),
// flip, measurement, accumulation.
constexpr int NPHASE = 5;
// A lattice of at least FOLD_MIN_TILES tiles has its measurement partials
// summed in FOLD_GROUPS groups on as many blocks before the accumulation.
constexpr int FOLD_MIN_TILES = 2048;
constexpr int FOLD_GROUPS = 64;

struct GraphEntry {
    int n;
    cudaGraphExec_t exec;
};

struct Engine {
    int R = 0, model = 0, prec = 0, start = 0;
    TileShape tile{1, 1, 1};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool use_graphs = true;
    std::vector<Rep> reps;      // host copy of the replica table
    std::vector<double> beta;   // current inverse temperature per replica
    Rep *d_reps = nullptr;
    Batch B;
    int64_t ntiles = 0, nblocks = 0;
    std::vector<void *> owned;
    std::vector<GraphEntry> graphs;
    uint64_t sweep = 0;
    uint64_t epoch = 0;  // host mirror of the device epoch (same for all replicas)
    uint64_t hst_epoch = 0;  // staging word of the initial epoch copy
    uint64_t launches = 0;
    bool labels_valid = false;

    // caller-owned device memory, if any: every array is carved from it
    // (256-byte aligned, in the order of workspace_bytes) and nothing is freed
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0, ws_used = 0;

    cudaError_t setup(int R, const int *Ls, const double *betas, int model, int prec, int start, double J,
                      const uint64_t *seeds, cudaStream_t user_stream, const TileShape &t, std::string &err,
                      void *workspace = nullptr, size_t workspace_bytes = 0);
    cudaError_t alloc(void **p, size_t bytes);
    void release();
    size_t spin_bytes(int r) const;
    cudaError_t set_beta(int r, double beta);
    cudaError_t sweeps(int n);
    cudaError_t measure();
    cudaError_t set_sweep(uint64_t s);
    cudaError_t set_trace(int r, int64_t cap);
    cudaError_t compute_labels();
    // mean device ms per sweep over n separately launched sweeps
    cudaError_t time_sweeps(int n, double &ms);
    cudaError_t guard_epoch(int n);
    int read_status(std::string &err);
    int launches_per_sweep() const;

    cudaError_t profile(int n, double *phase_ms);
    void enqueue_phase(int p, int mode);
    void enqueue_sweeps(int n);
    void enqueue_measure(int mode);
    cudaGraphExec_t graph_for(int n);
};

uint64_t ising_threshold(double beta, double J);

// Test hooks (pyro_debug_set): the next `fail_allocs` device allocations
// of an engine set-up report failure.
extern int g_fail_allocs;
// cudaMalloc behind the fail_allocs hook.
cudaError_t engine_malloc(void **p, size_t bytes);
// Test hook (pyro_debug_set): the crossing-link stamp that engines created
// from now on start at (0 by default), so that a test can take a chain
// across the stamps' wrap-around.
extern uint64_t g_epoch_start;
TileShape default_tile(const int *Ls, int R, int model);
// Device bytes of every array of a set of lattices (labels included), as
// the engine lays them out in a caller-owned workspace.
size_t workspace_bytes(int R, const int *Ls, int model, int prec, const TileShape &t);
std::string check_tile(const int *Ls, int R, int model, int prec, const TileShape &t);
size_t local_smem(int model, int prec, const TileShape &t);

}  // namespace pyro

struct pyro_ctx {
    pyro::Engine e;
};

struct pyro_batch_ctx {
    pyro::Engine e;
};
