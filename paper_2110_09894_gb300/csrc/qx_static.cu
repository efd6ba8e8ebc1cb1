// Contraction without any device allocation by the library or the caller's
// allocator: the workspace is a fixed array compiled into the library.
//
// Who needs this: host programs that cannot let a library allocate device
// memory -- applications that hand every byte of the GPU to their own pool
// allocator (so a cudaMalloc from a plugin fails or fragments their pool),
// and code that must not call cudaMalloc / cudaFree at all because those
// calls can synchronise the whole device.  Such callers pass device buffers
// for the bitstrings and amplitudes and nothing else.
//
// Cost: every GPU that loads libqx holds QX_STATIC_SCRATCH_BYTES of device
// memory for this array until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "qx.h"
#include "qx_internal.h"

static __device__ __align__(256) unsigned char g_qx_static_scratch[QX_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device, set on first use
}  // namespace

extern "C" int qx_contract_device_static(qx_handle h, const uint8_t* d_bits, int64_t n_bits, double* d_amps) {
    if (!h) return QX_EINVAL;
    const int dev = qx_internal_device(h);
    if (dev < 0) return qx_internal_fail(h, QX_ESTATE, "host-only handle has no device");
    if (dev >= kMaxDevices) return qx_internal_fail(h, QX_EINVAL, "device index beyond the static scratch table");
    if (cudaSetDevice(dev) != cudaSuccess) return qx_internal_fail(h, QX_ECUDA, "cudaSetDevice failed");
    void* addr = nullptr;
    {
        // In host code the array's name is only a host-side stand-in; the
        // device address comes from the runtime, once per device, with that
        // device current.
        std::lock_guard<std::mutex> g(g_lock);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_qx_static_scratch);
            if (e != cudaSuccess || !p)
                return qx_internal_fail(h, QX_ECUDA, "cudaGetSymbolAddress of the static scratch array failed");
            g_scratch_addr[dev] = p;
        }
        addr = g_scratch_addr[dev];
    }
    return qx_internal_contract_in(h, (char*)addr, QX_STATIC_SCRATCH_BYTES, d_bits, n_bits, d_amps);
}
