// Host-side call into the CUDA toolkit's own Philox4x32-10 (curand device
// API header, which carries a host code path).  Used only by the tests to
// pin the two independent Philox implementations of this repository against
// NVIDIA's library.
#define QUALIFIERS static inline
#include <vector_types.h>
#include <nv/target>
#include <curand_philox4x32_x.h>

extern "C" void curand_philox_ref(const unsigned* ctr, const unsigned* key, unsigned* out) {
  uint4 c;
  c.x = ctr[0]; c.y = ctr[1]; c.z = ctr[2]; c.w = ctr[3];
  uint2 k;
  k.x = key[0]; k.y = key[1];
  uint4 r = curand_Philox4x32_10(c, k);
  out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
}
