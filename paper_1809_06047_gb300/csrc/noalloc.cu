// alsub_refine_vertices_static: vertex refinement that allocates nothing.
//
// The ordinary alsub_refine_vertices keeps the positions of the intermediate levels in scratch
// memory that is either the caller's or the handle's own (allocated when the handle is made).
// This variant takes that scratch from a fixed array compiled into the library instead, so the
// call itself needs no device allocation at all: for callers that cannot call cudaMalloc at the
// point where they refine (code running inside another allocator's callback, or a host that
// forbids device allocation after start-up), and that cannot hand over a buffer of their own.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

// Holds the intermediate levels (two levels of float4 rows) of one call. Every GPU that loads the
// library keeps this array until the process exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" alsub_status alsub_refine_vertices_static(alsub_topology_t topo, const float *P0_dev,
                                                     float *PL_dev, void *stream) {
    if (!topo || !P0_dev || !PL_dev) return alsub::report(ALSUB_ERR_INVALID_ARG, "NULL argument");
    size_t need = 0;
    alsub_status st = alsub_refine_vertices_scratch_bytes(topo, &need);
    if (st != ALSUB_OK) return st;
    if (need > kStaticScratchBytes)
        return alsub::report(ALSUB_ERR_UNSUPPORTED,
                             "alsub_refine_vertices_static: the intermediate levels need more than the "
                             "32 MiB static scratch array; use alsub_refine_vertices");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return alsub::report(ALSUB_ERR_DEVICE, "alsub_refine_vertices_static: no usable current device");
    }
    void *scratch = nullptr;
    {
        // set-up, once per device, with that device current: the device address of the array
        // (its name in host code is only a host-side stand-in)
        std::lock_guard<std::mutex> g(g_lock);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return alsub::report(ALSUB_ERR_DEVICE, "alsub_refine_vertices_static: cudaGetSymbolAddress failed");
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    return alsub_refine_vertices(topo, P0_dev, PL_dev, scratch, stream);
}
