// noalloc.cu -- ifem_compute_forces_noalloc: element forces through the
// deterministic element-buffer path, with the per-element and per-node
// scratch taken from one file-scope device array instead of memory the
// library allocates. Compiled without FMA contraction.
#include <mutex>

#include "forces.cuh"
#include "handles.h"

namespace {

// Scratch: per-element nodal forces (12 reals per element), then per-node
// bending data (6 reals per node, 256-byte aligned). Every GPU that loads
// the library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_force_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

template <typename real>
cudaError_t launch(const DevBatch &b, const real *x, real *F, unsigned char *scratch, size_t bend_off,
                   unsigned long long *status, cudaStream_t s)
{
    real *ebuf = reinterpret_cast<real *>(scratch);
    real *bbuf = reinterpret_cast<real *>(scratch + bend_off);
    dim3 ge((b.max_elems + 255) / 256, b.n_inst), gn((b.max_nodes + 255) / 256, b.n_inst);
    // each launch is checked before the next is queued: a later kernel must
    // not read scratch that a failed launch never wrote, and the first error
    // is the one reported
    elem_force_kernel<real, false><<<ge, 256, 0, s>>>(b, x, nullptr, ebuf, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    node_gather_kernel<real><<<gn, 256, 0, s>>>(b, ebuf, F);
    if ((e = cudaGetLastError()) != cudaSuccess || !b.any_bending)
        return e;
    bend_pass1_kernel<real><<<gn, 256, 0, s>>>(b, x, bbuf);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    bend_pass2_kernel<real><<<gn, 256, 0, s>>>(b, x, bbuf, F);
    return cudaGetLastError();
}

}  // namespace

extern "C" int ifem_compute_forces_noalloc(ifem_ctx ctx, ifem_batch b, const void *x, void *F, void *stream)
{
    IFEM_DEVICE_SCOPE(ctx);
    if (!ctx || !b || b->ctx != ctx) {
        if (ctx)
            ctx->err = "compute_forces_noalloc: null or foreign batch";
        return IFEM_ERR_ARG;
    }
    if ((!x || !F) && b->N > 0) {
        ctx->err = "compute_forces_noalloc: null array";
        return IFEM_ERR_ARG;
    }
    const int dev = ctx->cfg.device;
    if (dev < 0 || dev >= kMaxDevices) {
        ctx->err = "compute_forces_noalloc: device ordinal above the supported 64";
        return IFEM_ERR_CAPACITY;
    }
    const size_t rs = ctx->cfg.precision == IFEM_FP64 ? sizeof(double) : sizeof(float);
    const size_t bend_off = align256((size_t)b->n_elems * 12 * rs);
    const size_t need = bend_off + (size_t)b->N * 6 * rs;
    if (need > kScratchBytes) {
        ctx->err = "compute_forces_noalloc: batch needs " + std::to_string(need) +
                   " bytes of scratch, above the fixed 33554432 (12 reals per element + 6 per node)";
        return IFEM_ERR_CAPACITY;
    }
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return IFEM_ERR_CUDA;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // host code only sees a stand-in for the device array: ask the
            // runtime for its address on this device, once
            e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_force_scratch);
            if (e != cudaSuccess) {
                g_scratch_ptr[dev] = nullptr;
                ctx->err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return IFEM_ERR_CUDA;
            }
        }
        scratch = g_scratch_ptr[dev];
    }
    if (b->inst.empty() || b->N == 0)
        return IFEM_OK;
    const DevBatch db = dev_batch(b);
    cudaStream_t s = (cudaStream_t)stream;
    e = ctx->cfg.precision == IFEM_FP64
            ? launch<double>(db, (const double *)x, (double *)F, (unsigned char *)scratch, bend_off, ctx->d_status, s)
            : launch<float>(db, (const float *)x, (float *)F, (unsigned char *)scratch, bend_off, ctx->d_status, s);
    if (e != cudaSuccess) {
        ctx->err = std::string("compute_forces_noalloc: ") + cudaGetErrorString(e);
        return IFEM_ERR_CUDA;
    }
    return IFEM_OK;
}
