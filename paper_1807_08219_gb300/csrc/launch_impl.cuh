// launch_impl.cuh -- host-side launch sequences, instantiated once per
// precision (kernels_f32.cu with FMA contraction, kernels_f64.cu without).
#pragma once
#include <type_traits>

#include "common.cuh"
#include "forces.cuh"
#include "transfer.cuh"
#include "lagrangian.cuh"

namespace ifem {

#define IFEM_LAUNCH_CHECK()                      \
    do {                                         \
        cudaError_t e_ = cudaGetLastError();     \
        if (e_ != cudaSuccess)                   \
            return e_;                           \
    } while (0)

template <typename real>
cudaError_t forces_impl(const ForcesArgs &a)
{
    const DevBatch &b = a.b;
    if (b.n_inst == 0)
        return cudaSuccess;
    const real *x = (const real *)a.x;
    real *F = (real *)a.F;
    cudaStream_t s = a.stream;
    if constexpr (std::is_same<real, float>::value) {
        if (!a.hvp && a.scatter == 1 && b.fused_ok) {
        size_t sm = fused_smem_bytes(b.max_nodes);
        const int n = a.inst_n > 0 ? a.inst_n : b.n_inst;
        if (a.inst0 < 0 || a.inst0 + n > b.n_inst)
            return cudaErrorInvalidValue;
        cudaFuncSetAttribute(forces_fused_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        forces_fused_f32_kernel<<<n, 512, sm, s>>>(b, (const float *)a.x, (float *)a.F, a.w.status, a.inst0);
        IFEM_LAUNCH_CHECK();
        return cudaSuccess;
        }
    }
    if (a.inst0 != 0 || (a.inst_n != 0 && a.inst_n != b.n_inst))
        return cudaErrorInvalidValue;   // particle ranges: the one-CTA-per-particle kernel only
    dim3 blk(256);
    dim3 ge((b.max_elems + 255) / 256, b.n_inst);
    dim3 gn((b.max_nodes + 255) / 256, b.n_inst);
    real *ebuf = (real *)a.w.elem_buf;
    if (a.hvp)
        elem_force_kernel<real, true><<<ge, blk, 0, s>>>(b, x, (const real *)a.wv, ebuf, a.w.status);
    else
        elem_force_kernel<real, false><<<ge, blk, 0, s>>>(b, x, nullptr, ebuf, a.w.status);
    IFEM_LAUNCH_CHECK();
    node_gather_kernel<real><<<gn, blk, 0, s>>>(b, ebuf, F);
    IFEM_LAUNCH_CHECK();
    if (!a.hvp && b.any_bending) {
        real *bb = (real *)a.w.bend_buf;
        bend_pass1_kernel<real><<<gn, blk, 0, s>>>(b, x, bb);
        IFEM_LAUNCH_CHECK();
        bend_pass2_kernel<real><<<gn, blk, 0, s>>>(b, x, bb, F);
        IFEM_LAUNCH_CHECK();
    }
    return cudaSuccess;
}

template <typename real>
cudaError_t bin_impl(const TransferArgs &a, int det_sort, int with_cand, int stages)
{
    const DevBatch &b = a.b;
    const DevWork &w = a.w;
    const long long nt = a.g.n_tiles;
    cudaStream_t s = a.stream;
    const long long no = nt * kOwnSub3;
    if (with_cand && stages != BIN_ALL)
        return cudaErrorInvalidValue;
    const bool empty = b.n_inst == 0 || b.N == 0;
    dim3 gn((b.max_nodes + 255) / 256, b.n_inst);
    // one-pass binning of the FP32 halo path: kBinPer nodes per thread
    dim3 g1((b.max_nodes + 256 * kBinPer - 1) / (256 * kBinPer), b.n_inst);
    if (stages & BIN_COUNT) {
        if (with_cand)
            cudaMemsetAsync(w.cand_count, 0, sizeof(int) * (nt + 1), s);
        // own counts, then (FP32 halo path) the per-tile flags and |F| sums behind them
        cudaMemsetAsync(w.own_count, 0, sizeof(int) * (no + 1 + (with_cand ? 0 : 4 * nt)), s);
        cudaMemsetAsync(w.counters, 0, sizeof(int) * kCounters, s);
        IFEM_LAUNCH_CHECK();
        if (empty)
            return cudaSuccess;
        if (with_cand) {
            bin_kernel<real, false><<<gn, 256, 0, s>>>(b, a.g, w, (const real *)a.x);
        } else {
            if constexpr (!std::is_same<real, float>::value)
                return cudaErrorInvalidValue;   // the one-pass own lists are FP32 only
            else
                own_count_kernel<<<g1, 256, 0, s>>>(b, a.g, w, (const float *)a.x);
        }
        IFEM_LAUNCH_CHECK();
        int nb = (int)((no + kScanBlock - 1) / kScanBlock);
        // without candidate lists the local own offsets go to the cursors, and
        // own_scatter_kernel writes the final offsets beside them
        scan_local_kernel<<<nb, kScanThreads, 0, s>>>(with_cand ? nt : 0, no, w.cand_count, w.own_count, w.cand_off,
                                                      with_cand ? w.own_off : w.own_cursor, w.scan_blocks,
                                                      w.counters + 8, w.counters + 4);
        IFEM_LAUNCH_CHECK();
    }
    if (empty || !(stages & BIN_PLACE))
        return cudaSuccess;
    if (with_cand) {
        scan_finish_kernel<<<(unsigned)((no + 1 + 255) / 256), 256, 0, s>>>(nt, no, w);
        IFEM_LAUNCH_CHECK();
        bin_kernel<real, true><<<gn, 256, 0, s>>>(b, a.g, w, (const real *)a.x);
        IFEM_LAUNCH_CHECK();
    } else {
        // enough threads for every tile boundary as well as every node
        const long long per_inst = ((nt + 1 + 255) / 256 + b.n_inst - 1) / b.n_inst;
        dim3 gs((unsigned)std::max<long long>(g1.x, per_inst), b.n_inst);
        own_scatter_kernel<<<gs, 256, 0, s>>>(b, w, nt, (const float *)a.F);
        IFEM_LAUNCH_CHECK();
    }
    if (det_sort) {
        sort_segments_kernel<<<a.n_sm * 4, 512, 0, s>>>(w);
        IFEM_LAUNCH_CHECK();
    }
    if constexpr (std::is_same<real, double>::value) {
        if (a.kernel == 0 && w.wtab) {
            det_weights_kernel<<<(unsigned)((3 * b.N + 255) / 256), 256, 0, s>>>(b, a.g, w.wtab, (const double *)a.x);
            IFEM_LAUNCH_CHECK();
        }
    }
    return cudaSuccess;
}

template <typename real>
cudaError_t spread_impl(const TransferArgs &a)
{
    const DevBatch &b = a.b;
    cudaStream_t s = a.stream;
    // the fused halo transfer right after its binning: own_scatter_kernel
    // cleared the per-tile sums and the binning the work counter
    const bool cleared = a.binned && a.halo && a.u != nullptr && a.v != nullptr;
    if (!cleared)
        cudaMemsetAsync(a.w.red_tile, 0, sizeof(double) * 3 * a.g.n_tiles, s);
    IFEM_LAUNCH_CHECK();
    if (b.n_inst == 0 || b.N == 0)
        return cudaSuccess;
    if constexpr (std::is_same<real, float>::value) {
        const int E = a.g.max_edge;
        if (!cleared)
            cudaMemsetAsync(a.w.counters + 2, 0, sizeof(int), s);
        if (a.halo) {
            // with u and v given, interpolation is fused into the spread, and
            // with xn also the position update
            const bool fused = a.u != nullptr && a.v != nullptr;
            if (fused && a.halo == 2) {
                auto kp = a.xn ? transfer_staged_kernel<true> : transfer_staged_kernel<false>;
                const size_t sm = (size_t)pair_smem_bytes(E);
                cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                int occ = 1;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kp, kStagedThreads, sm);
                occ = occ < 1 ? 1 : occ;
                if (!a.pdl) {
                    kp<<<a.n_sm * occ, kStagedThreads, sm, s>>>(b, a.g, a.w, (const float *)a.x,
                                                              (const float *)a.F, (float *)a.f, a.density,
                                                              (const float *)a.u, (float *)a.v, (const float *)a.vp,
                                                              (float *)a.xn, (float)a.dt, a.lattice);
                    IFEM_LAUNCH_CHECK();
                    return cudaSuccess;
                }
                // programmatic dependent launch: the CTAs of this grid may start once
                // every CTA of the previous kernel in the stream has signalled
                // (griddepcontrol.launch_dependents, at its start); they read
                // nothing it writes
                cudaLaunchConfig_t cfg{};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                attr[0].val.programmaticStreamSerializationAllowed = 1;
                cfg.gridDim = dim3(a.n_sm * occ);
                cfg.blockDim = dim3(kStagedThreads);
                cfg.dynamicSmemBytes = sm;
                cfg.stream = s;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                return cudaLaunchKernelEx(&cfg, kp, b, a.g, a.w, (const float *)a.x, (const float *)a.F,
                                          (float *)a.f, a.density, (const float *)a.u, (float *)a.v,
                                          (const float *)a.vp, (float *)a.xn, (float)a.dt, a.lattice);
            }
            auto kern = !fused ? spread_halo_kernel<false>
                               : (a.xn ? spread_halo_kernel<true, true> : spread_halo_kernel<true>);
            size_t sm = sizeof(int) * (size_t)halo_ints(E);
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            int occ = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, sm);
            occ = occ < 1 ? 1 : occ;
            kern<<<a.n_sm * occ, 256, sm, s>>>(b, a.g, a.w, (const float *)a.x, (const float *)a.F, (float *)a.f,
                                               a.density, (const float *)a.u, (float *)a.v,
                                               (const float *)a.vp, (float *)a.xn, (float)a.dt);
            IFEM_LAUNCH_CHECK();
            return cudaSuccess;
        }
        size_t acc = a.acc64 ? sizeof(long long) : sizeof(int);
        size_t sm = acc * 3 * (size_t)acc_stride(E, E, E);
        auto kern = a.kernel == 0 ? (a.acc64 ? spread_fast_kernel<0, long long> : spread_fast_kernel<0, int>)
                                  : (a.acc64 ? spread_fast_kernel<1, long long> : spread_fast_kernel<1, int>);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, sm);
        occ = occ < 1 ? 1 : occ;
        kern<<<a.n_sm * occ, 256, sm, s>>>(b, a.g, a.w, (const float *)a.x, (const float *)a.F, (float *)a.f,
                                           a.density, (float)a.support);
    } else {
        if (a.kernel == 0) {
            // warp per (tile, lattice) over the binning's stencil table
            if (!a.w.wtab)
                return cudaErrorInvalidValue;
            // as many warps per CTA (up to kDetWarps) as the largest tile's
            // accumulators fit in one CTA's shared memory
            const size_t per_warp = det_warp_bytes(a.g.max_edge);
            const int warps = (int)std::min<size_t>(kDetWarps, kMaxCtaSmemBytes / per_warp);
            if (warps < 1)
                return cudaErrorInvalidValue;
            const size_t sm = per_warp * warps;
            cudaFuncSetAttribute(spread_det_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            int occ = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spread_det_warp_kernel, 32 * warps, sm);
            occ = occ < 1 ? 1 : occ;
            spread_det_warp_kernel<<<a.n_sm * occ, 32 * warps, sm, s>>>(b, a.g, a.w, (const double *)a.F,
                                                                      (double *)a.f, a.density);
            IFEM_LAUNCH_CHECK();
            return cudaSuccess;
        }
        auto kern = spread_det_mls_kernel;
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kDetThreads, 0);
        occ = occ < 1 ? 1 : occ;
        kern<<<a.n_sm * occ, kDetThreads, 0, s>>>(b, a.g, a.w, (const double *)a.x, (const double *)a.F,
                                                  (double *)a.f, a.density, a.support);
    }
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t interp_impl(const TransferArgs &a)
{
    const DevBatch &b = a.b;
    if (b.n_inst == 0 || b.N == 0)
        return cudaSuccess;
    if constexpr (std::is_same<real, float>::value) {
        unsigned grid = (unsigned)((3 * b.N + 255) / 256);
        if (a.kernel == 0)
            interp_direct_kernel<0><<<grid, 256, 0, a.stream>>>(b, a.g, a.w, (const float *)a.u, (const float *)a.x,
                                                               (float *)a.v, (float)a.support);
        else
            interp_direct_kernel<1><<<grid, 256, 0, a.stream>>>(b, a.g, a.w, (const float *)a.u, (const float *)a.x,
                                                               (float *)a.v, (float)a.support);
    } else {
        unsigned grid = (unsigned)((b.N + 255) / 256);
        if (a.kernel == 0)
            interp_kernel<real, true, 0><<<grid, 256, 0, a.stream>>>(b, a.g, a.w, (const real *)a.u,
                                                                    (const real *)a.x, (real *)a.v, (real)a.support, 0,
                                                                    a.use_wtab && a.w.wtab != nullptr);
        else
            interp_kernel<real, true, 1><<<grid, 256, 0, a.stream>>>(b, a.g, a.w, (const real *)a.u,
                                                                    (const real *)a.x, (real *)a.v, (real)a.support, 0,
                                                                    0);
    }
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t reduce_impl(const ReduceArgs &a)
{
    const int parts = a.parts ? a.parts : 3;
    const unsigned blocks = (unsigned)(a.b.n_inst + ((parts & 2) ? 3 * a.g.n_boxes : 0));
    if (blocks == 0)
        return cudaSuccess;
    reduce_kernel<real><<<blocks, kReduceThreads, 0, a.stream>>>(a.b, a.g, a.w.red_tile, (const real *)a.x,
                                                               (const real *)a.F, (const real *)a.v, a.red, parts);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t fluid_impl(const FluidArgs &a)
{
    const DevBatch &b = a.b;
    if (b.n_inst == 0)
        return cudaSuccess;
    dim3 blk(256);
    dim3 ge((b.max_elems + 255) / 256, b.n_inst);
    dim3 gn((b.max_nodes + 255) / 256, b.n_inst);
    real *ebuf = (real *)a.w.elem_buf;
    fluid_elem_kernel<real><<<ge, blk, 0, a.stream>>>(b, (const real *)a.x, (const real *)a.u, (const real *)a.C,
                                                      (real)a.eta, (real)a.cp, ebuf);
    IFEM_LAUNCH_CHECK();
    if (a.add)
        fluid_gather_kernel<real, true><<<gn, blk, 0, a.stream>>>(b, ebuf, (real *)a.F);
    else
        fluid_gather_kernel<real, false><<<gn, blk, 0, a.stream>>>(b, ebuf, (real *)a.F);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t interp_cc_impl(const TransferArgs &a, int ncomp)
{
    const DevBatch &b = a.b;
    if (b.n_inst == 0 || b.N == 0)
        return cudaSuccess;
    unsigned grid = (unsigned)((b.N * ncomp + 255) / 256);
    if (a.kernel == 0)
        interp_cc_kernel<real, 0><<<grid, 256, 0, a.stream>>>(b, a.g, a.w, (const real *)a.u, ncomp,
                                                              (const real *)a.x, (real *)a.v, (real)a.support);
    else
        interp_cc_kernel<real, 1><<<grid, 256, 0, a.stream>>>(b, a.g, a.w, (const real *)a.u, ncomp,
                                                              (const real *)a.x, (real *)a.v, (real)a.support);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t ab2_impl(const LagrangeArgs &a)
{
    const long long n3 = 3 * a.b.N;
    if (n3 == 0)
        return cudaSuccess;
    ab2_kernel<real><<<(unsigned)((n3 + 255) / 256), 256, 0, a.stream>>>(
        n3, (const real *)a.x, (real *)(a.x_out ? a.x_out : a.x), (const real *)a.v, (const real *)a.vp,
        (real)a.dt);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t volume_impl(const LagrangeArgs &a)
{
    if (a.b.n_inst == 0)
        return cudaSuccess;
    volume_kernel<real><<<a.b.n_inst, kVolThreads, 0, a.stream>>>(a.b, (const real *)a.x, a.out);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t vcorr_impl(const LagrangeArgs &a)
{
    if (a.b.n_inst == 0)
        return cudaSuccess;
    dim3 gn((a.b.max_nodes + 255) / 256, a.b.n_inst);
    vc_alpha_kernel<real><<<gn, 256, 0, a.stream>>>(a.b, (const real *)a.x, a.alpha);
    IFEM_LAUNCH_CHECK();
    vc_correct_kernel<real><<<a.b.n_inst, kVolThreads, 0, a.stream>>>(a.b, (real *)a.x, a.alpha, a.V0, a.out,
                                                                       a.status);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

template <typename real>
cudaError_t area_normals_impl(const DevBatch &b, const void *x, void *nA, cudaStream_t s)
{
    if (b.n_inst == 0)
        return cudaSuccess;
    dim3 gn((b.max_nodes + 255) / 256, b.n_inst);
    area_normal_kernel<real><<<gn, 256, 0, s>>>(b, (const real *)x, (real *)nA);
    IFEM_LAUNCH_CHECK();
    return cudaSuccess;
}

}  // namespace ifem
