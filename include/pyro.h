/*
 * pyro.h -- C ABI of libpyro: Swendsen-Wang multi-cluster sweeps of the
 * ferromagnetic Ising, classical XY and classical Heisenberg models on the
 * periodic pyrochlore lattice, on one GB300 GPU (sm_103a).
 *
 * The physics is that of Soldatov, Nefedev, Komura and Okabe, "Large-scale
 * calculation of ferromagnetic spin systems on the pyrochlore lattice"
 * (arXiv:1612.08312):
 *   Sec. 2  lattice: L x L x L cubic cells of 16 sites, periodic boundaries,
 *           N = 16 L^3 sites, coordination number six;
 *   Eq. 1   H = -J sum_<ij> s_i . s_j, unit n-vectors, n = 1 (Ising),
 *           2 (XY), 3 (Heisenberg);
 *   Sec. 2  Swendsen-Wang multi-cluster update on one GPU, with Wolff's
 *           embedded cluster (reflection about a random plane) for n = 2, 3;
 *   Eq. 2   moment ratio U = <m^4>/<m^2>^2 with m = M/N.
 *
 * Conventions the paper leaves open, fixed here so that a run is a
 * deterministic function of (L, model, start, seed, beta sequence):
 *   site index   i = 16 (x + L (y + L z)) + 4 f + mu, position (quarter
 *                cell units) 4 (x,y,z) + A_f + B_mu, A = {0,(0,2,2),(2,0,2),
 *                (2,2,0)}, B = {0,(0,1,1),(1,0,1),(1,1,0)};
 *   bond id      the bonds of cell c are numbered b = 48 c + 16 g + 4 f + q,
 *                f the FCC point of the tetrahedron, (g, q) = (0,0) up
 *                pair (0,1), (0,1) up (1,2), (0,2) up (2,3), (0,3) up (0,3),
 *                (1,0) up (0,2), (1,1) up (1,3), (1,2) down (0,2), (1,3) down
 *                (1,3), (2,0) down (0,1), (2,1) down (1,2), (2,2) down (2,3),
 *                (2,3) down (0,3) (pairs of basis vertices);
 *   random bits  Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 *                (j_lo, j_hi, sweep, tag); tags 1 bond, 2 flip, 3 axis,
 *                4 initial state (sweep field 0xFFFFFFFF), 5 tie.  A call's
 *                128 bits are read as 16 bytes (byte t: bits 8 (t & 3).. of
 *                output word t >> 2), 4 words, or 128 bits (bit t: bit t & 31
 *                of output word t >> 5);
 *   bond uniform w_b = (byte b & 15 of bond call b >> 4) << 24 | (low 24
 *                bits of word b & 3 of tie call b >> 2); the tie bits are
 *                only needed when the top bytes of w_b and the threshold are
 *                equal;
 *   Ising bond   active iff s_i = s_j and w_b < floor((1 - exp(-2 beta J))
 *                2^32);
 *   n-vector     axis r drawn once per sweep; active iff p_i p_j > 0 and
 *                w_b < floor((1 - exp(-2 beta J p_i p_j)) 2^32), p_i = s_i.r;
 *   cluster      canonical label = minimum site index in the cluster; the
 *                cluster flips iff bit (label) of the flip stream is 1;
 *                n-vector flip s <- s - 2 (s.r) r, then s <- s/|s|;
 *   measurement  after every sweep: E, m = |M|/N, m2 = m m, m4 = m2 m2,
 *                accumulated in FP64 with Neumaier compensation.
 *
 * Error behaviour: every int-returning call returns PYRO_OK (0) or a
 * negative PYRO_E_* code and sets a thread-local message readable with
 * pyro_last_error().  No C++ exception crosses this interface.  Calls on
 * one handle are not thread-safe; different handles are independent.
 * Work is enqueued on the handle's CUDA stream; calls that return data to
 * the host synchronise that stream first.  Device-side failures (a union-
 * find or barrier wait that exceeded its bound) are recorded in a device
 * status word and returned by the next synchronising call as
 * PYRO_E_NOCONVERGE or PYRO_E_TIMEOUT.
 */
#ifndef PYRO_H
#define PYRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pyro_ctx *pyro_handle;
typedef struct pyro_batch_ctx *pyro_batch;

enum { PYRO_ISING = 1, PYRO_XY = 2, PYRO_HEIS = 3 };
enum { PYRO_FP32 = 0, PYRO_FP64 = 1 };
enum { PYRO_START_UP = 0, PYRO_START_RANDOM = 1 };

enum {
    PYRO_OK = 0,
    PYRO_E_INVAL = -1,      /* bad argument: L out of range, model, beta < 0 or NaN, n < 0, NULL */
    PYRO_E_NOMEM = -2,      /* device or host allocation failed */
    PYRO_E_CUDA = -3,       /* a CUDA runtime call failed (message has the CUDA error) */
    PYRO_E_NOCONVERGE = -4, /* a union-find loop exceeded its iteration bound */
    PYRO_E_TIMEOUT = -5,    /* a grid barrier wait exceeded its time bound */
    PYRO_E_STATE = -6       /* call not valid in the current state */
};

/* Largest supported lattice: labels are int32 and N = 16 L^3 < 2^31. */
#define PYRO_MAX_L 511

typedef struct {
    int L;             /* cells per edge, 1 <= L <= PYRO_MAX_L */
    int model;         /* PYRO_ISING, PYRO_XY or PYRO_HEIS */
    int precision;     /* n-vector spins: PYRO_FP32 or PYRO_FP64 (ignored for Ising) */
    int start;         /* PYRO_START_UP (all +1 / e_x) or PYRO_START_RANDOM */
    double J;          /* ferromagnetic coupling, J > 0 (the paper uses J = 1) */
    uint64_t seed;     /* Philox key */
    void *stream;      /* cudaStream_t to run on; NULL = the library creates one */
    int tile[3];       /* labelling tile in cells: power-of-two edges, each dividing L, at most
                          512 cells; {0,0,0} = default (Ising 8 x 8 x 4, n-vector 8 x 4 x 4,
                          each edge reduced to the largest power of two dividing L) */
    void *workspace;   /* NULL = the library allocates (and frees) the lattice's device memory;
                          else caller-owned device memory (for instance a torch tensor's data_ptr),
                          at least pyro_workspace_bytes(cfg) bytes, 256-byte aligned, from which
                          every device array of the lattice is carved; the library frees none of
                          it, and it must stay valid until pyro_destroy.  It opens with the
                          statistics record, padded to 256 bytes; the spins follow at byte 256
                          in the layout of pyro_get_state */
    size_t workspace_bytes; /* size of workspace in bytes */
} pyro_config;

typedef struct {
    uint64_t count;    /* sweeps accumulated since the last reset */
    double sum_E;      /* sum of E over those sweeps (Neumaier-compensated FP64) */
    double sum_E2;     /* sum of E^2 */
    double sum_m2;     /* sum of m^2 */
    double sum_m4;     /* sum of m^4 */
    double sum_absm;   /* sum of |m| */
} pyro_stats_t;

/* ---- single lattice ------------------------------------------------------ */

/* Create a lattice with J = 1, FP32 n-vector spins, ordered start, a
 * library-owned stream and the default tile.  *out receives the handle,
 * owned by the caller until pyro_destroy.  Sec. 2 (lattice), Eq. 1. */
int pyro_init(pyro_handle *out, int L, int model, uint64_t seed);

/* Same with every option of pyro_config.  cfg is read, not kept.  With a
 * workspace, PYRO_E_NOMEM if it is smaller than pyro_workspace_bytes(cfg),
 * PYRO_E_INVAL if it is not 256-byte aligned; no device allocation is made
 * (pyro_set_trace alone allocates its ring buffer). */
int pyro_init_ex(pyro_handle *out, const pyro_config *cfg);

/* Device bytes of a lattice created with cfg (its spins, tile-local labels,
 * crossing-cluster links, flip words, face masks, statistics, canonical
 * labels, partial sums and replica record; Sec. 2 lattice of N = 16 L^3
 * sites), for a caller that owns the device memory and passes it in
 * cfg->workspace.  cfg->workspace itself is ignored.  0 if cfg is invalid
 * (pyro_last_error says why). */
size_t pyro_workspace_bytes(const pyro_config *cfg);

/* Enqueue n Swendsen-Wang sweeps at inverse temperature beta (Sec. 2) on
 * the handle's stream; each sweep is followed by the measurement of Eq. 2,
 * accumulated into the statistics.  Asynchronous: returns after enqueueing.
 * beta >= 0 and finite, n >= 0. */
int pyro_sweep(pyro_handle h, double beta, int n);

/* Instantaneous E, m^2, m^4 of the current configuration (Eq. 1, Eq. 2).
 * Synchronises the stream.  Any pointer may be NULL. */
int pyro_measure(pyro_handle h, double *E, double *m2, double *m4);

/* Accumulated statistics since the last reset (Eq. 2 moments and energy).
 * Synchronises the stream. */
int pyro_stats(pyro_handle h, pyro_stats_t *s);
int pyro_reset_stats(pyro_handle h);

/* Spins in canonical site order, host memory, synchronous.
 * Ising: N int8 values +1/-1 (bytes = N).  n-vector: N x n doubles,
 * site-major (bytes = 8 n N); the FP32 store rounds them to float.
 * bytes must equal the exact size. */
int pyro_get_spins(pyro_handle h, void *host, size_t bytes);
int pyro_set_spins(pyro_handle h, const void *host, size_t bytes);

/* The library's compact device layout of the spins, copied to/from host
 * memory (pinned memory gives full bandwidth):
 *   Ising:   one uint16 per cell, bit (i & 15) of word (i >> 4) is 1 iff
 *            s_i = -1 (bytes = N / 8);
 *   n-vector: n component planes of N floats (FP32) or doubles (FP64).
 * pyro_state_bytes gives the size.  Enqueued on the handle's stream; the
 * host buffer must stay valid until the stream is synchronised. */
size_t pyro_state_bytes(pyro_handle h);
int pyro_get_state(pyro_handle h, void *host, size_t bytes);
int pyro_set_state(pyro_handle h, const void *host, size_t bytes);

/* Canonical cluster labels of the last sweep (the minimum site index of
 * each site's cluster), N int32 values, computed on demand from the sweep's
 * tile-local labels (the first call allocates a 4 N byte buffer).
 * PYRO_E_STATE if the spins were set since the last sweep.  Synchronises. */
int pyro_get_labels(pyro_handle h, int32_t *host, size_t bytes);

/* Sweep counter: the sweep field of the Philox counter of the next sweep. */
int pyro_get_sweep(pyro_handle h, uint64_t *sweep);
int pyro_set_sweep(pyro_handle h, uint64_t sweep);

/* Per-sweep trace: keep the last `capacity` sweeps' (E, m2, m4, M_x)
 * records in a device ring buffer (0 disables).  pyro_get_trace copies the
 * most recent min(count, capacity) records, oldest first, as 4 doubles
 * each, and returns their number through *n. */
int pyro_set_trace(pyro_handle h, int64_t capacity);
int pyro_get_trace(pyro_handle h, double *host, int64_t max_records, int64_t *n);

/* Wait for all enqueued work; report any device-side status. */
int pyro_sync(pyro_handle h);

/* Facts about a handle. */
int64_t pyro_num_sites(pyro_handle h);
int pyro_get_tile(pyro_handle h, int tile[3]);
void *pyro_get_stream(pyro_handle h);

/* Number of kernel launches this handle has issued (for accounting). */
uint64_t pyro_launch_count(pyro_handle h);

/* Whether multi-sweep calls replay captured CUDA graphs (default on; only
 * with a library-owned stream).  Off = one launch per phase per sweep. */
int pyro_set_graphs(pyro_handle h, int on);

/* Autotuner: equilibrate a scratch lattice for 60 sweeps at beta, then
 * replay the same nsweeps sweeps from that state with every candidate
 * labelling tile (power-of-two edges dividing L, 64 to 512 cells) and
 * return the fastest in tile_out (pass it in pyro_config.tile) and its
 * device ms per sweep (NULL allowed).  Results are cached per (GPU
 * name, L, model, precision) in the process and, if the environment
 * variable PYRO_AUTOTUNE_CACHE names a file, across processes.  Allocates
 * and frees a scratch lattice per candidate; synchronises the device. */
int pyro_autotune(int L, int model, int precision, double beta, int nsweeps, int tile_out[3], double *ms_per_sweep);

/* Test hooks for failure handling, process-wide:
 *   PYRO_DEBUG_FAIL_ALLOCS  the next `value` device allocations made while
 *                           creating a lattice or batch report failure
 *                           (the call returns PYRO_E_NOMEM, nothing leaks);
 *   PYRO_DEBUG_UNITE_BOUND  iteration bound of one shared-memory union
 *                           (default 4096; 0 makes every union give up at
 *                           once, so the next synchronising call returns
 *                           PYRO_E_NOCONVERGE);
 *   PYRO_DEBUG_NOALLOC_STAMP  the stamp of the crossing-cluster links of the
 *                           next pyro_ising_sweep_noalloc call on the current
 *                           device (32-bit value), so that a test can take
 *                           the calls across the stamps' wrap-around;
 *   PYRO_DEBUG_EPOCH_START  the stamp that lattices and batches created from
 *                           now on start their crossing-cluster links at
 *                           (32-bit value; default 0), likewise. */
enum { PYRO_DEBUG_FAIL_ALLOCS = 1, PYRO_DEBUG_UNITE_BOUND = 2, PYRO_DEBUG_NOALLOC_STAMP = 3,
       PYRO_DEBUG_EPOCH_START = 4 };
int pyro_debug_set(int key, int64_t value);

/* Tracing: run n sweeps at beta like pyro_sweep, but as separate launches
 * bracketed by CUDA events, and return the mean device time in ms of each
 * of the five phases of a sweep in phase_ms[0..4]: tile-local labelling
 * (with bond activation), unions of clusters crossing tile faces, flip,
 * measurement, accumulation.  Synchronises.  The chain advances exactly as
 * with pyro_sweep. */
#define PYRO_NPHASE 5
int pyro_profile_phases(pyro_handle h, double beta, int n, double *phase_ms);

void pyro_destroy(pyro_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char *pyro_last_error(void);

/* ---- sweep without allocation ------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory: a sweep embedded in an application whose
 * framework owns the device memory budget through its own caching
 * allocator, a plugin that may not allocate after start-up, or a latency-
 * sensitive loop in which cudaMalloc/cudaFree would synchronise the device
 * and stall other streams.
 *
 * One Ising Swendsen-Wang sweep, the same chain step as pyro_sweep on a
 * lattice with this seed and sweep counter (same conventions as above),
 * with every input and output supplied by the caller and all scratch memory
 * (flip bits, tile-crossing bond masks, per-block partial sums, the lattice
 * record and its statistics, the tile-local labels, the links between
 * clusters that cross tile faces) taken from one file-scope device array of
 * PYRO_NOALLOC_SCRATCH_BYTES bytes.  That array exists on every GPU that
 * loads the library and stays there until the process exits.
 *
 *   spins_in   device, L^3 uint16 in the compact layout of pyro_get_state
 *   spins_out  device, L^3 uint16: the spins after the sweep; either equal
 *              to spins_in (an in-place update) or not overlapping it, else
 *              PYRO_E_INVAL
 *   labels     device, 16 L^3 int32: canonical cluster labels of the sweep
 *   meas       device, 4 doubles: E, m^2, m^4 and M of the new configuration
 *   L          1 <= L <= PYRO_NOALLOC_MAX_L, else PYRO_E_INVAL
 *   beta, seed, sweep   inverse temperature (J = 1), Philox key, sweep field
 *   stream     cudaStream_t to run on (NULL = the legacy default stream)
 *
 * Calls no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it.  Every
 * call on a device uses the same array, which keeps the previous call's
 * contents; the call re-initialises what must start from zero.  Calls whose
 * work overlaps on the GPU (other streams, other host threads) race on the
 * array and must be serialised by the caller.  Synchronises the stream
 * before returning, and returns PYRO_E_NOCONVERGE if a union-find loop hit
 * its bound. */
#define PYRO_NOALLOC_MAX_L 32
#define PYRO_NOALLOC_SCRATCH_BYTES 6488576
int pyro_ising_sweep_noalloc(const uint16_t *spins_in, uint16_t *spins_out, int32_t *labels, double *meas,
                             int L, double beta, uint64_t seed, uint64_t sweep, void *stream);

/* ---- batched replicas ----------------------------------------------------- */

/* R independent lattices of sizes L[r] at inverse temperatures beta[r],
 * one model and precision, updated together: every phase of a sweep is one
 * launch over all replicas' tiles, and a multi-sweep call is a CUDA graph.
 * Replica r uses seed + r * 0x9E3779B97F4A7C15 (mod 2^64), so it is the
 * same chain as a single lattice created with that seed.  start as in
 * pyro_config.  Independent runs (Sec. 2: five independent runs). */
int pyro_batch_init(pyro_batch *out, int R, const int *L, const double *beta, int model,
                    int precision, int start, uint64_t seed);

/* Same with a labelling tile for every replica (power-of-two edges dividing
 * every L; NULL or {0,0,0} = the default of the lattices' common divisor),
 * e.g. from pyro_batch_autotune. */
int pyro_batch_init_ex(pyro_batch *out, int R, const int *L, const double *beta, int model,
                       int precision, int start, uint64_t seed, const int tile[3]);

/* Autotuner for a batch: equilibrates R replicas (sizes L, inverse
 * temperatures beta) with the default tile for 60 sweeps, then replays the
 * same nsweeps sweeps with every candidate tile and returns the fastest in
 * tile_out and its device ms per batch sweep.  Cached per (GPU name, the set
 * of distinct L, model, precision) like pyro_autotune.  Allocates and frees
 * scratch batches; synchronises. */
int pyro_batch_autotune(int R, const int *L, const double *beta, int model, int precision, int nsweeps,
                        int tile_out[3], double *ms_per_sweep);
int pyro_batch_sweep(pyro_batch b, int n);
int pyro_batch_stats(pyro_batch b, int r, pyro_stats_t *s);
/* Every replica's statistics in s[0 .. R) and every replica's instantaneous
 * E, m^2, m^4 in out[3 r + 0..2], each with one device-to-host copy (the
 * replicas' records are contiguous on the device).  Synchronise. */
int pyro_batch_stats_all(pyro_batch b, pyro_stats_t *s);
int pyro_batch_measure_all(pyro_batch b, double *out);
int pyro_batch_reset_stats(pyro_batch b);
int pyro_batch_measure(pyro_batch b, int r, double *E, double *m2, double *m4);
int pyro_batch_get_spins(pyro_batch b, int r, void *host, size_t bytes);
int pyro_batch_sync(pyro_batch b);
int64_t pyro_batch_total_sites(pyro_batch b);
void *pyro_batch_get_stream(pyro_batch b);
uint64_t pyro_batch_launch_count(pyro_batch b);
void pyro_batch_destroy(pyro_batch b);

/* ---- generic lattices: a bond list, a neighbour table or the simple-cubic
 *      lattice, optionally diluted ------------------------------------------
 *
 * Sec. 2: the SW program needs only the table of every site's nearest
 * neighbours, so the same sweep runs on any lattice given as a list of
 * bonds.  Sec. 3.4 (Eq. 5-6) compares with the simple-cubic lattice (also
 * coordination six); Sec. 4 names diluted lattices as the extension.
 *
 * Conventions (the pyrochlore ones above, with these changes):
 *   bond id      bond e of the list joins sites bond_i[e] and bond_j[e]; its
 *                random-number id is e, its uniform w_e as above.  Listing
 *                the pyrochlore bonds in the order of their ids above gives
 *                the pyrochlore chain of the same seed, bit for bit;
 *   simple cubic L^3 sites, site i = x + L (y + L z), bond 3 i + d joins i
 *                to the next site along axis d (periodic), L >= 2;
 *   dilution     a vacant site takes no part: bonds touching it are absent,
 *                it is a cluster of its own and never flips; a bond with mask
 *                0 is absent; absent bonds are never active and are left out
 *                of E;
 *   measurement  E = -J sum over present bonds of s_i . s_j, m = |M| / N_occ,
 *                M summed over occupied sites (m = 0 if none is occupied).
 * Errors, streams and statistics as for pyro_handle. */
typedef struct pyro_graph_ctx *pyro_graph;

typedef struct {
    int model;                /* PYRO_ISING, PYRO_XY or PYRO_HEIS */
    int precision;            /* n-vector spins: PYRO_FP32 or PYRO_FP64 (ignored for Ising) */
    int start;                /* PYRO_START_UP or PYRO_START_RANDOM (per site as for pyro_handle) */
    double J;                 /* ferromagnetic coupling, J > 0 */
    uint64_t seed;            /* Philox key */
    void *stream;             /* cudaStream_t; NULL = the library creates one */
    int sc_L;                 /* > 0: the simple-cubic sc_L^3 lattice (2 <= sc_L <= 1290), bonds
                                 implicit; bond_i, bond_j must then be NULL */
    int64_t nsites;           /* sc_L = 0: number of sites N, 1 <= N < 2^31 */
    int64_t nbonds;           /* sc_L = 0: number of bonds, 0 <= nbonds < 2^35 */
    const int32_t *bond_i;    /* sc_L = 0: host, nbonds sites in [0, N) */
    const int32_t *bond_j;    /* sc_L = 0: host, nbonds sites in [0, N), bond_j[e] != bond_i[e] */
    const uint8_t *site_mask; /* host, N bytes, 0 = vacant; NULL = every site occupied */
    const uint8_t *bond_mask; /* host, one byte per bond, 0 = absent; NULL = every bond present */
} pyro_graph_config;

/* Create a generic lattice; the host arrays are read, not kept (the bond
 * list is copied to the device).  PYRO_E_INVAL on a bad argument (a site
 * out of range, a self-loop, sizes out of range). */
int pyro_graph_init(pyro_graph *out, const pyro_graph_config *cfg);

/* Bond list of a neighbour table nbr (N rows of z entries, -1 = none;
 * Sec. 2): slot (i, k) with i < nbr[i z + k] is a bond, in the order of
 * (i, k).  Returns the number of bonds and, if bond_i and bond_j are not
 * NULL, writes them; PYRO_E_INVAL if an entry is out of range or names its
 * own row, or if j does not appear in i's row as often as i in j's row.
 * Host only; no GPU is needed. */
int64_t pyro_graph_bonds_from_table(int64_t N, int z, const int32_t *nbr, int32_t *bond_i, int32_t *bond_j);

/* n sweeps at inverse temperature beta (as pyro_sweep). */
int pyro_graph_sweep(pyro_graph g, double beta, int64_t n);
/* E, m^2, m^4 of the current configuration.  Synchronises. */
int pyro_graph_measure(pyro_graph g, double *E, double *m2, double *m4);
int pyro_graph_stats(pyro_graph g, pyro_stats_t *s);
int pyro_graph_reset_stats(pyro_graph g);
/* Spins in site order: Ising int8 +-1 (N bytes); n-vector doubles, site-
 * major (8 n N bytes).  Vacant sites' spins are kept and returned as well. */
int pyro_graph_get_spins(pyro_graph g, void *host, size_t bytes);
int pyro_graph_set_spins(pyro_graph g, const void *host, size_t bytes);
/* Canonical cluster labels of the last sweep (N int32; before the first
 * sweep every site is its own cluster). */
int pyro_graph_get_labels(pyro_graph g, int32_t *host, int64_t n);
/* The sweep counter that keys the next sweep's random numbers (as
 * pyro_set_sweep / pyro_get_sweep; the get synchronises and returns 0 for a
 * NULL handle or a failed read). */
int pyro_graph_set_sweep(pyro_graph g, uint64_t sweep);
uint64_t pyro_graph_get_sweep(pyro_graph g);
/* Sites and bonds of the lattice (0 for a NULL handle). */
int64_t pyro_graph_num_sites(pyro_graph g);
int64_t pyro_graph_num_bonds(pyro_graph g);
/* Wait for the handle's work; PYRO_E_NOCONVERGE if a union hit its bound. */
int pyro_graph_sync(pyro_graph g);
void *pyro_graph_get_stream(pyro_graph g);
/* Kernel launches issued so far (four per Ising sweep, five for n > 1,
 * two per pyro_graph_measure, one at creation). */
uint64_t pyro_graph_launch_count(pyro_graph g);
/* Free the lattice's device memory (after its stream's work) and the handle. */
void pyro_graph_destroy(pyro_graph g);

#ifdef __cplusplus
}
#endif

#endif /* PYRO_H */
