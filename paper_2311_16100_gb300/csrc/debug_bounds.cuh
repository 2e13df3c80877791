// Range checks of computed memory indices for the debug variant of the
// library (compiled with -DCS_DEBUG_BOUNDS; in the normal build CS_IN is the
// constant true and costs nothing).  A failing check skips the access it
// guards and sets a flag of its translation unit; cs_check_device_status
// reads and clears every unit's flag and reports CS_ERR_INTERNAL.  Nothing
// faults or traps, and the context stays usable.
#pragma once

#include <cuda_runtime.h>

namespace cs {

#ifdef CS_DEBUG_BOUNDS

// host side: each translation unit registers the reader of its flag
void dbg_register(unsigned (*reader)());

namespace {

__device__ unsigned int g_dbg_bad;   // this translation unit's flag

__device__ __forceinline__ bool dbg_in_range(long long i, long long n) {
  if ((unsigned long long)i < (unsigned long long)n) return true;
  atomicOr(&g_dbg_bad, 1u);
  return false;
}

// reads the current device's copy of the flag and clears it
unsigned dbg_read_and_clear() {
  unsigned v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_dbg_bad, sizeof v) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v && cudaMemcpyToSymbol(g_dbg_bad, &z, sizeof z) != cudaSuccess) cudaGetLastError();
  return v;
}

struct DbgRegistrar {
  DbgRegistrar() { dbg_register(dbg_read_and_clear); }
};
DbgRegistrar g_dbg_registrar;

}  // namespace

#define CS_IN(i, n) (::cs::dbg_in_range((long long)(i), (long long)(n)))

#else

#define CS_IN(i, n) true

#endif

}  // namespace cs
