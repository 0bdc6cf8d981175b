// kernels_f32.cu -- FP32 instantiation of the libifem kernels (FMA allowed).
#include "launch_impl.cuh"

namespace ifem {
cudaError_t launch_forces_f32(const ForcesArgs &a) { return forces_impl<float>(a); }
cudaError_t launch_bin_f32(const TransferArgs &a, int det_sort, int with_cand, int stages)
{
    return bin_impl<float>(a, det_sort, with_cand, stages);
}
cudaError_t launch_spread_f32(const TransferArgs &a) { return spread_impl<float>(a); }
cudaError_t launch_interp_f32(const TransferArgs &a) { return interp_impl<float>(a); }
cudaError_t launch_reduce_f32(const ReduceArgs &a) { return reduce_impl<float>(a); }
cudaError_t launch_fluid_f32(const FluidArgs &a) { return fluid_impl<float>(a); }
cudaError_t launch_interp_cc_f32(const TransferArgs &a, int ncomp) { return interp_cc_impl<float>(a, ncomp); }
cudaError_t launch_ab2_f32(const LagrangeArgs &a) { return ab2_impl<float>(a); }
cudaError_t launch_volume_f32(const LagrangeArgs &a) { return volume_impl<float>(a); }
cudaError_t launch_vcorr_f32(const LagrangeArgs &a) { return vcorr_impl<float>(a); }
cudaError_t launch_area_normals_f32(const DevBatch &b, const void *x, void *nA, cudaStream_t s)
{
    return area_normals_impl<float>(b, x, nA, s);
}
}  // namespace ifem
