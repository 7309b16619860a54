// Host-side runner for cuRAND's Philox4x32-10 block function, compiled from
// the cuRAND device header for the host.  Used only by the oracle pin that
// checks the oracle's Philox against an independent implementation.
#define QUALIFIERS static inline __host__ __device__
#include <curand_kernel.h>
#include <stdint.h>

extern "C" void curand_philox_blocks(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    for (int i = 0; i < n; ++i) {
        uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
        uint4 r = curand_Philox4x32_10(c, k);
        out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
    }
}
