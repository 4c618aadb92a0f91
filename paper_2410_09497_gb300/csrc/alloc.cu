// Every device and pinned-host allocation of the library goes through these
// functions.  They carry a host-side fault injector for the failure-path
// tests: with STK_FAIL_ALLOC_AFTER=N in the environment, the first N
// allocations succeed and every later one fails with cudaErrorMemoryAllocation
// (nothing is allocated); the count restarts whenever the variable's value
// changes and the injector is off when it is unset or empty.  Only the
// allocation call is faked; no GPU work is affected.
#include <cstdlib>
#include <mutex>
#include <string>

#include "internal.h"

namespace stk {

namespace {

std::mutex g_mu;
std::string g_armed;  // value of STK_FAIL_ALLOC_AFTER the count belongs to
long g_count = 0;

bool injected_failure() {
  const char* v = std::getenv("STK_FAIL_ALLOC_AFTER");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!v || !*v) {
    g_armed.clear();
    g_count = 0;
    return false;
  }
  if (g_armed != v) {
    g_armed = v;
    g_count = 0;
  }
  return ++g_count > std::strtol(v, nullptr, 10);
}

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

cudaError_t dev_alloc_async(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, s);
}

cudaError_t host_alloc_pinned(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocHost(p, bytes);
}

}  // namespace stk
