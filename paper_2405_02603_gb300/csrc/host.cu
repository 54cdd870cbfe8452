// host.cu -- pinned host buffers placed on the host NUMA node nearest the
// GPU, for the host-buffer solves (fsp_solve_host, fsp_solve_host_many).
//
// On a Grace-based node the host memory of each CPU is its own NUMA node and
// the GPU reaches one of them directly over NVLink-C2C; a staging buffer that
// the first-touch policy happened to place on another node crosses the
// CPU-to-CPU link on every copy.  fsp_host_alloc maps anonymous memory, binds
// it to the requested node (mbind), touches every page, and page-locks it
// for the device (cudaHostRegister).
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <cerrno>
#include <cstdint>
#include <cstring>

#include "../../include/fsp.h"

namespace {

constexpr int kMpolBind = 2;  // MPOL_BIND of the Linux memory-policy API

bool bind_to_node(void *p, size_t bytes, int node) {
#ifdef SYS_mbind
    if (node < 0 || node >= 1024) return false;
    unsigned long mask[1024 / (8 * sizeof(unsigned long))] = {};
    mask[node / (8 * sizeof(unsigned long))] |= 1ul << (node % (8 * sizeof(unsigned long)));
    return syscall(SYS_mbind, p, bytes, kMpolBind, mask, (unsigned long)1024, 0u) == 0;
#else
    (void)p, (void)bytes, (void)node;
    return false;
#endif
}

}  // namespace

extern "C" {

int fsp_device_host_numa(int device) {
    int v = -1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrHostNumaId, device) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return v;
}

fsp_status fsp_host_alloc(void **out, size_t bytes, int numa_node) {
    if (!out || bytes == 0) return FSP_EINVAL;
    *out = nullptr;
    void *p = mmap(nullptr, bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (p == MAP_FAILED) return FSP_ENOMEM;
    if (numa_node >= 0 && !bind_to_node(p, bytes, numa_node)) {
        munmap(p, bytes);
        return FSP_EUNSUPPORTED;
    }
    std::memset(p, 0, bytes);  // place every page now, under the binding
    if (cudaHostRegister(p, bytes, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(p, bytes);
        return FSP_ECUDA;
    }
    *out = p;
    return FSP_OK;
}

fsp_status fsp_host_free(void *p, size_t bytes) {
    if (!p) return FSP_EINVAL;
    const cudaError_t e = cudaHostUnregister(p);
    if (e != cudaSuccess) cudaGetLastError();
    munmap(p, bytes);
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

}  // extern "C"
