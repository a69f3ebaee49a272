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

#define NSP_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      if (e_ == cudaErrorMemoryAllocation)                                                \
        throw ::nsp::Error(NSP_ERR_OOM, std::string(#call) + ": " + cudaGetErrorString(e_)); \
      throw ::nsp::Error(NSP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    }                                                                                     \
  } while (0)

// Every kernel launch of the library passes through this check, which also counts it.
int64_t count_launch();
#define NSP_LAUNCH_CHECK()             \
  do {                                 \
    ::nsp::count_launch();             \
    NSP_CUDA(cudaGetLastError());      \
  } while (0)

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

}  // namespace nsp
