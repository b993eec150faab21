// Error reporting and version of the C ABI.
#include <atomic>
#include <cstdio>
#include <string>

#include "internal.h"

namespace chns {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void note_launches_undo(unsigned long long k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
unsigned long long chns_launches_now() { return g_launches.load(); }

void set_error(const std::string& msg) { g_last_error = msg; }

chns_status cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  g_last_error = buf;
  return e == cudaErrorMemoryAllocation ? CHNS_ENOMEM : CHNS_ECUDA;
}

}  // namespace chns

extern "C" const char* chns_last_error(void) { return chns::g_last_error.c_str(); }

extern "C" const char* chns_version(void) { return "chns-gb300 0.1 (sm_103a)"; }

extern "C" uint64_t chns_kernel_launches(void) { return chns::g_launches.load(); }
