// host_buffer.cpp -- page-locked host buffers for the host copies of
// stencil_run_host (a library service; the paper has none).
//
// stencil_host_alloc maps anonymous memory aligned to 2 MiB, asks the kernel
// for transparent huge pages (madvise(MADV_HUGEPAGE): fewer translations for
// the copy engine), touches every page and registers the range with CUDA
// (cudaHostRegister, portable).  Whatever the page size, GPU copies of host
// pages the CPU has not touched for a few seconds run slowly on Grace-based
// machines; stencil_run_host touches its buffers right before each copy
// (run.cu).
#include <sys/mman.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>

#include <cuda_runtime.h>

#include "internal.h"
#include "launch.h"

namespace gbs {
namespace {

constexpr size_t kHuge = (size_t)2 << 20;

struct Mapping {
    void *base;
    size_t length;
};

std::mutex g_host_mu;
std::map<uintptr_t, Mapping> g_host_buffers;  // user pointer -> mapping

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" stencil_status stencil_host_alloc(void **ptr, size_t bytes)
try {
    if (!ptr) return fail(STENCIL_ERR_INVALID_ARG, "stencil_host_alloc: ptr is null");
    *ptr = nullptr;
    if (bytes == 0) return fail(STENCIL_ERR_INVALID_ARG, "stencil_host_alloc: bytes is 0");
    const size_t size = (bytes + kHuge - 1) / kHuge * kHuge;
    const size_t length = size + kHuge;  // room to align the start to 2 MiB
    void *base = mmap(nullptr, length, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (base == MAP_FAILED) return fail(STENCIL_ERR_OOM, "stencil_host_alloc: mmap failed");
    const uintptr_t a = (reinterpret_cast<uintptr_t>(base) + kHuge - 1) / kHuge * kHuge;
    void *p = reinterpret_cast<void *>(a);
    madvise(p, size, MADV_HUGEPAGE);  // advice only: without huge pages the buffer still works
    std::memset(p, 0, size);          // back every page before it is registered
    cudaError_t e = cudaHostRegister(p, size, cudaHostRegisterPortable);
    if (e != cudaSuccess) {
        munmap(base, length);
        return cuda_fail(e, "stencil_host_alloc: cudaHostRegister");
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        g_host_buffers[a] = Mapping{base, length};
    }
    *ptr = p;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_host_alloc");
}

extern "C" stencil_status stencil_host_free(void *ptr)
try {
    if (!ptr) return STENCIL_OK;
    Mapping m{};
    {
        std::lock_guard<std::mutex> lock(g_host_mu);
        auto it = g_host_buffers.find(reinterpret_cast<uintptr_t>(ptr));
        if (it == g_host_buffers.end())
            return fail(STENCIL_ERR_INVALID_ARG, "stencil_host_free: not a pointer from stencil_host_alloc");
        m = it->second;
        g_host_buffers.erase(it);
    }
    cudaError_t e = cudaHostUnregister(ptr);
    munmap(m.base, m.length);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "stencil_host_free: cudaHostUnregister");
} catch (...) {
    return gbs::abi_exception("stencil_host_free");
}
