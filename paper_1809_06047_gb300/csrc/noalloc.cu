// alsub_refine_vertices_static: vertex refinement that allocates nothing.
//
// The ordinary alsub_refine_vertices keeps the positions of the intermediate levels in scratch
// memory that is either the caller's or the handle's own (allocated when the handle is made), and
// a call that repeats the previous call's pointers is captured into a CUDA graph (a private stream,
// graph instantiation). This variant takes its scratch from a fixed array compiled into the
// library and launches its kernels directly on the caller's stream, so after its first call on a
// device it makes no device allocation of any kind: for callers that cannot allocate at the point
// where they refine (code running inside another allocator's callback, or a host that forbids
// device allocation after start-up) and that cannot hand over a buffer of their own.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

// Holds the intermediate levels (two levels of float4 rows) of one call. The array lives in this
// file's module: the driver reserves it on a device when the module is loaded there, which the
// set-up below forces, and it stays reserved until the process exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {};

// Set-up, once per device, with that device current: the device address of the array (its name in
// host code is only a host-side stand-in and must never reach a kernel).
alsub_status scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            if (e == cudaErrorMemoryAllocation)
                return alsub::report(ALSUB_ERR_OOM, "alsub_refine_vertices_static: no device memory for the "
                                                    "32 MiB static scratch array");
            return alsub::report(ALSUB_ERR_DEVICE, "alsub_refine_vertices_static: cudaGetSymbolAddress failed");
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ALSUB_OK;
}

}  // namespace

extern "C" alsub_status alsub_refine_vertices_static(alsub_topology_t topo, const float *P0_dev,
                                                     float *PL_dev, void *stream) {
    if (!topo || !P0_dev || !PL_dev) return alsub::report(ALSUB_ERR_INVALID_ARG, "NULL argument");
    alsub::TopoImpl &T = *alsub::topology_impl(topo);
    if (T.scratch_bytes > kStaticScratchBytes)
        return alsub::report(ALSUB_ERR_UNSUPPORTED,
                             "alsub_refine_vertices_static: the intermediate levels need more than the "
                             "32 MiB static scratch array; use alsub_refine_vertices");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return alsub::report(ALSUB_ERR_DEVICE, "alsub_refine_vertices_static: no usable current device");
    }
    // the array is per device: the topology's arrays must live on the current device, or its
    // kernels would be handed another GPU's copy of the array
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, T.status) != cudaSuccess) {
        cudaGetLastError();
        return alsub::report(ALSUB_ERR_DEVICE, "alsub_refine_vertices_static: cannot locate the topology's device");
    }
    if (a.device != dev)
        return alsub::report(ALSUB_ERR_INVALID_ARG, "alsub_refine_vertices_static: the topology lives on another "
                                                    "device than the current one");
    void *scratch = nullptr;
    alsub_status st = scratch_address(dev, &scratch);
    if (st != ALSUB_OK) return st;
    return alsub::refine_direct(T, P0_dev, PL_dev, scratch, (cudaStream_t)stream);
}
