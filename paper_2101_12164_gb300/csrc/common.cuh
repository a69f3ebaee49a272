// Shared helpers of the CUDA translation units: error propagation, device buffers,
// launch geometry and the device error word.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/nsp.h"

namespace nsp {

// An exception carrying an nsp_status; every C entry point catches it.
struct Error : std::runtime_error {
  nsp_status status;
  Error(nsp_status s, const std::string &msg) : std::runtime_error(msg), status(s) {}
};

#define NSP_STR2_(x) #x
#define NSP_STR_(x) NSP_STR2_(x)
#define NSP_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      const std::string m_ = std::string(#call " at " __FILE__ ":" NSP_STR_(__LINE__) ": ") + \
                             cudaGetErrorString(e_);                                        \
      throw ::nsp::Error(e_ == cudaErrorMemoryAllocation ? NSP_ERR_OOM : NSP_ERR_CUDA, m_);   \
    }                                                                                       \
  } while (0)

// Every kernel launch of the library passes through this check, which also counts it.
int64_t count_launch();
int64_t launches_counted();
void add_launches(int64_t k);
#define NSP_LAUNCH_CHECK()             \
  do {                                 \
    ::nsp::count_launch();             \
    NSP_CUDA(cudaGetLastError());      \
  } while (0)

// Message of the last failed C call on this thread (nsp_last_error).
void set_last_error(const char *msg);

inline void require(bool ok, nsp_status s, const char *msg) {
  if (!ok) throw Error(s, msg);
}

// Device-side status word written by kernels (first error wins). Codes:
enum DevErr : int32_t {
  DEV_OK = 0,
  DEV_NOT_SPD = 1,      // aux = factor block id
  DEV_BREAKDOWN = 2,    // aux = 0
  DEV_TIMEOUT = 3,      // aux = where
  DEV_BAD_INDEX = 4,
};
struct DevStatus {
  int32_t code;
  int32_t aux;
};

__device__ inline void dev_fail(DevStatus *st, int32_t code, int32_t aux) {
  if (atomicCAS(&st->code, 0, code) == 0) st->aux = aux;
}

// RAII device allocation.
template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) NSP_CUDA(cudaMalloc(&p, count * sizeof(T)));
  }
  void ensure(size_t count) { if (count > n) alloc(count); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void upload(const std::vector<T> &h, cudaStream_t st) {
    alloc(h.size());
    if (!h.empty()) NSP_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  }
  size_t bytes() const { return n * sizeof(T); }
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Opt a kernel into `bytes` of dynamic shared memory when its static plus dynamic shared
// memory exceed the default 48 KB window (the attribute only ever grows).
template <typename K>
inline void ensure_dyn_smem(K kernel, size_t bytes) {
  if (bytes == 0) return;
  cudaFuncAttributes fa{};
  NSP_CUDA(cudaFuncGetAttributes(&fa, kernel));
  if (fa.sharedSizeBytes + bytes > 48 * 1024 && (size_t)fa.maxDynamicSharedSizeBytes < bytes)
    NSP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace nsp
