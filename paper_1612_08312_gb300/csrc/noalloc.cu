// noalloc.cu -- an Ising sweep entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code embedded in a host application
// whose framework owns the whole device memory budget through its own
// caching allocator, plugins that are forbidden to allocate after start-up,
// and latency-sensitive loops in which cudaMalloc / cudaFree would
// synchronise the device and stall every other stream.  They pass their
// inputs and outputs in, and the sweep's scratch memory (flip bits, tile-
// crossing bond masks, per-block partial sums, the replica record and its
// statistics, the tile-local labels, the crossing-cluster links) lives in
// the file-scope device array below instead of in library allocations.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "engine.h"

namespace pyro {

void ising_launch_phase(int p, const Batch &B, int64_t ntiles, cudaStream_t s);
void launch_labels(const Batch &B, int64_t ntiles, cudaStream_t s);
void ising_launch_measure(const Batch &B, int64_t ntiles, cudaStream_t s);
cudaError_t ising_prepare(const TileShape &t);
void launch_accumulate(const Batch &B, bool ising, int mode, int nc, cudaStream_t s);
void set_error(const std::string &msg);

namespace {

constexpr int64_t NA_MAX_CELLS = (int64_t)PYRO_NOALLOC_MAX_L * PYRO_NOALLOC_MAX_L * PYRO_NOALLOC_MAX_L;
constexpr int64_t NA_MAX_SITES = 16 * NA_MAX_CELLS;
constexpr int64_t NA_MAX_TILES = NA_MAX_CELLS;  // 1-cell tiles at worst
// Byte offsets inside the scratch array (each 256-byte aligned).
constexpr size_t NA_OFF_REP = 0;
constexpr size_t NA_OFF_STATS = 256;
constexpr size_t NA_OFF_F = 512;
constexpr size_t NA_OFF_DMASK = NA_OFF_F + (size_t)NA_MAX_CELLS * sizeof(uint16_t);
constexpr size_t NA_OFF_PARTIALS = NA_OFF_DMASK + (size_t)NA_MAX_CELLS * sizeof(uint32_t);
constexpr size_t NA_OFF_L16 = NA_OFF_PARTIALS + (size_t)NA_MAX_TILES * 4 * sizeof(double);
constexpr size_t NA_OFF_P = NA_OFF_L16 + (size_t)NA_MAX_SITES * sizeof(uint16_t);
constexpr size_t NA_BYTES = NA_OFF_P + (size_t)NA_MAX_SITES * sizeof(unsigned long long);
static_assert(sizeof(Rep) <= 256 && sizeof(DevStats) <= 256, "scratch header slots too small");
static_assert(NA_BYTES == PYRO_NOALLOC_SCRATCH_BYTES, "scratch size differs from the header");

// The scratch memory, held by every device that loads the library.
static __device__ __align__(256) unsigned char na_scratch[NA_BYTES];

// Device address of na_scratch per device ordinal, found once per device,
// and the stamp of the next call's crossing-cluster links on that device.
// The array starts zeroed, so stamps start at 1.
constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
void *na_addr[NA_MAX_DEVICES] = {};
uint32_t na_epoch[NA_MAX_DEVICES] = {};

__global__ void na_setup_kernel(Rep rep, Rep *rep_slot, DevStats *st, unsigned long long sweep, uint32_t epoch)
{
    *rep_slot = rep;
    DevStats z = {};
    z.sweep = sweep;
    z.epoch = epoch;
    z.last_epoch = epoch;  // the labels of this call use this call's links
    *st = z;
}

}  // namespace

// Test hook (pyro_debug_set): the stamp of the next call's links on the
// current device, so that a test can take the calls across the stamps'
// wrap-around.
int noalloc_set_stamp(uint32_t stamp)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return -1;
    std::lock_guard<std::mutex> lock(na_mutex);
    na_epoch[dev] = stamp;
    return 0;
}

namespace {

int na_fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

}  // namespace
}  // namespace pyro

using namespace pyro;

extern "C" int pyro_ising_sweep_noalloc(const uint16_t *spins_in, uint16_t *spins_out, int32_t *labels,
                                        double *meas, int L, double beta, uint64_t seed, uint64_t sweep,
                                        void *stream)
{
    if (!spins_in || !spins_out || !labels || !meas) return na_fail(PYRO_E_INVAL, "NULL argument");
    if (L < 1 || L > PYRO_NOALLOC_MAX_L)
        return na_fail(PYRO_E_INVAL, "pyro_ising_sweep_noalloc: L must be in [1, " +
                                         std::to_string(PYRO_NOALLOC_MAX_L) + "] (fixed scratch size)");
    if (!(beta >= 0.0) || !std::isfinite(beta)) return na_fail(PYRO_E_INVAL, "beta must be finite and >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(PYRO_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(PYRO_E_INVAL, "device ordinal out of range");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int Ls[1] = {L};
    const TileShape t = default_tile(Ls, 1, PYRO_ISING);
    const int nt = t.TX * t.TY * t.TZ;
    unsigned char *base = nullptr;
    uint32_t epoch = 0;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, na_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(PYRO_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = ising_prepare(t);
            if (e != cudaSuccess) return na_fail(PYRO_E_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
            na_addr[dev] = p;
        }
        base = static_cast<unsigned char *>(na_addr[dev]);
        if (na_epoch[dev] >= 0xFFFFFFF0u) {
            // stamps would wrap: mark every link as stale again
            e = cudaMemsetAsync(base + NA_OFF_P, 0, (size_t)NA_MAX_SITES * sizeof(unsigned long long), s);
            if (e != cudaSuccess) return na_fail(PYRO_E_CUDA, std::string("scratch reset: ") + cudaGetErrorString(e));
            na_epoch[dev] = 0;
        }
        epoch = ++na_epoch[dev];
    }

    Rep rep = {};
    rep.spins = spins_out;
    rep.P = reinterpret_cast<unsigned long long *>(base + NA_OFF_P);
    rep.labels = labels;
    rep.L16 = reinterpret_cast<uint16_t *>(base + NA_OFF_L16);
    rep.F = reinterpret_cast<uint16_t *>(base + NA_OFF_F);
    rep.dmask = reinterpret_cast<uint32_t *>(base + NA_OFF_DMASK);
    rep.st = reinterpret_cast<DevStats *>(base + NA_OFF_STATS);
    rep.seed = seed;
    rep.thr = ising_threshold(beta, 1.0);
    rep.K2 = 2.0 * beta;
    rep.J = 1.0;
    rep.ncells = (int64_t)L * L * L;
    rep.N = 16 * rep.ncells;
    rep.L = L;
    rep.ntx = L / t.TX;
    rep.nty = L / t.TY;

    Batch B;
    std::memset(&B, 0, sizeof(B));
    B.reps = reinterpret_cast<const Rep *>(base + NA_OFF_REP);
    B.partials = reinterpret_cast<double *>(base + NA_OFF_PARTIALS);
    B.R = 1;
    B.TX = t.TX;
    B.TY = t.TY;
    B.TZ = t.TZ;
    while ((1 << B.lTX) < t.TX) ++B.lTX;
    while ((1 << B.lTY) < t.TY) ++B.lTY;
    while ((1 << B.lTZ) < t.TZ) ++B.lTZ;
    const int64_t ntiles = rep.ncells / nt;
    B.tile_begin[1] = ntiles;
    B.block_begin[1] = (rep.ncells + CELL_BLOCK - 1) / CELL_BLOCK;

    if (spins_in != spins_out) {
        const size_t nb = (size_t)rep.ncells * sizeof(uint16_t);
        const uintptr_t a = reinterpret_cast<uintptr_t>(spins_in), b = reinterpret_cast<uintptr_t>(spins_out);
        if (a < b + nb && b < a + nb)
            return na_fail(PYRO_E_INVAL, "pyro_ising_sweep_noalloc: spins_in and spins_out overlap without being equal");
        e = cudaMemcpyAsync(spins_out, spins_in, nb, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return na_fail(PYRO_E_CUDA, std::string("spin copy: ") + cudaGetErrorString(e));
    }
    na_setup_kernel<<<1, 1, 0, s>>>(rep, reinterpret_cast<Rep *>(base + NA_OFF_REP), rep.st, sweep, epoch);
    for (int p = 0; p < 3; ++p) ising_launch_phase(p, B, ntiles, s);
    ising_launch_measure(B, ntiles, s);
    launch_accumulate(B, true, 2, 1, s);
    launch_labels(B, ntiles, s);
    e = cudaMemcpyAsync(meas, rep.st->last, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(PYRO_E_CUDA, std::string("sweep launch: ") + cudaGetErrorString(e));
    int status = 0;
    e = cudaMemcpyAsync(&status, &rep.st->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(PYRO_E_CUDA, std::string("sweep: ") + cudaGetErrorString(e));
    if (status & ST_NOCONVERGE) return na_fail(PYRO_E_NOCONVERGE, "union-find exceeded its iteration bound");
    return PYRO_OK;
}
