// Host-side call of cuRAND's Philox4x32-10 (from the CUDA toolkit header),
// used by the CPU tests as an implementation independent of the oracle's.
#define QUALIFIERS static inline
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

extern "C" void probe_philox(const unsigned *ctr, const unsigned *key, unsigned *out, long n)
{
    for (long t = 0; t < n; ++t) {
        uint4 c = make_uint4(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]);
        uint2 k = make_uint2(key[2 * t], key[2 * t + 1]);
        uint4 o = curand_Philox4x32_10(c, k);
        out[4 * t] = o.x; out[4 * t + 1] = o.y; out[4 * t + 2] = o.z; out[4 * t + 3] = o.w;
    }
}
