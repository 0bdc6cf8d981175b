// kernels_f64.cu -- FP64 deterministic instantiation of the libifem kernels.
// Compiled with --fmad=false: every multiply and add rounds separately, in
// the evaluation order written in the kernels, so results are bit-identical
// to a plain IEEE FP64 evaluation of the same expressions.
#include "launch_impl.cuh"

namespace ifem {
cudaError_t launch_forces_f64(const ForcesArgs &a) { return forces_impl<double>(a); }
cudaError_t launch_bin_f64(const TransferArgs &a, int det_sort, int with_cand, int stages)
{
    return bin_impl<double>(a, det_sort, with_cand, stages);
}
cudaError_t launch_spread_f64(const TransferArgs &a) { return spread_impl<double>(a); }
cudaError_t launch_interp_f64(const TransferArgs &a) { return interp_impl<double>(a); }
cudaError_t launch_reduce_f64(const ReduceArgs &a) { return reduce_impl<double>(a); }
cudaError_t launch_fluid_f64(const FluidArgs &a) { return fluid_impl<double>(a); }
cudaError_t launch_interp_cc_f64(const TransferArgs &a, int ncomp) { return interp_cc_impl<double>(a, ncomp); }
cudaError_t launch_ab2_f64(const LagrangeArgs &a) { return ab2_impl<double>(a); }
cudaError_t launch_volume_f64(const LagrangeArgs &a) { return volume_impl<double>(a); }
cudaError_t launch_vcorr_f64(const LagrangeArgs &a) { return vcorr_impl<double>(a); }
cudaError_t launch_area_normals_f64(const DevBatch &b, const void *x, void *nA, cudaStream_t s)
{
    return area_normals_impl<double>(b, x, nA, s);
}
}  // namespace ifem
