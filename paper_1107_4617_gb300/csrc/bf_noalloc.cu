// bf_backward_noalloc: the adjoint pass for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: a plugin running inside a host
// application that owns every byte of the GPU's memory through its own pool
// and forbids libraries from allocating, or a latency-critical loop where an
// allocation's implicit device synchronisation is not acceptable. They can
// pass inputs and outputs they already own, but not the workspace
// bf_backward needs for its per-CTA dL/dsigma_r partial sums. This entry
// point keeps that scratch in a fixed array compiled into the library
// instead.
//
// The array lives in file-scope device memory: every GPU that loads the
// library holds it (BF_NOALLOC_MAX_PARTIALS floats) until the process exits.
// Host code cannot pass the array's name to a kernel: on the host that name
// is only a stand-in, not a device address. Its device address on the current
// device is looked up with cudaGetSymbolAddress on every call (a host-side
// lookup that allocates nothing). Looking it up each time, rather than once
// per device, keeps the address right after a cudaDeviceReset, which
// destroys the device's context and can reload the module elsewhere.
#include "bf_internal.cuh"
#include "bf_trace.cuh"

namespace {

// Fixed scratch for the per-CTA partial sums (and, for harmonic chunks, the two
// image-sized accumulators); no entry needs to start at zero, because each
// call writes every slot it later reads.
__device__ __align__(256) float g_noalloc_partials[BF_NOALLOC_MAX_PARTIALS];

// Device address of the scratch array on the current device.
bf_status scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return bf::set_cuda_error(e);
    *out = p;
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_backward_noalloc(const void* img, const float* out,
                                         const float* grad_out, const void* saved, int H, int W,
                                         int r, float sigma_r, float T, int N, float* grad_img,
                                         float* grad_sigma, const bf_opts* opts, void* stream) {
    BF_TRACE("bf_backward_noalloc");
    const size_t cap = sizeof(float) * (size_t)BF_NOALLOC_MAX_PARTIALS;
    const size_t need = bf_backward_workspace_bytes(H, W, r, sigma_r, T, N, opts);
    if (need > cap) return BF_ERR_UNSUPPORTED;  // call needs more scratch than the array holds
    void* scratch = nullptr;
    bf_status st = scratch_address(&scratch);
    if (st != BF_OK) return st;
    return bf_backward(img, out, grad_out, saved, H, W, r, sigma_r, T, N, grad_img, grad_sigma,
                       scratch, cap, opts, stream);
}
