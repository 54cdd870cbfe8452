// plane_f32.cu -- host launchers of the fused plane passes (plane.cuh),
// single precision, N = 64, 128, 256.
#include "plane.cuh"

namespace fsp {
namespace fast {
namespace {

template <typename T, int N> cudaError_t launch_plane_n(bool fwd, const PlaneArgs &a, cudaStream_t s) {
    using K = PlaneCfg<T, N>;
    using G = PlaneGeo<T, N>;
    auto kern = fwd ? k_plane_fwd<T, N> : k_plane_inv<T, N>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(N * K::C));  // one cluster of C CTAs per z-plane
    cfg.blockDim = dim3((unsigned)G::NTH);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K::C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T> cudaError_t launch_plane(bool fwd, int N, const PlaneArgs &a, cudaStream_t s) {
    switch (N) {
    case 64: return launch_plane_n<T, 64>(fwd, a, s);
    case 128: return launch_plane_n<T, 128>(fwd, a, s);
    case 256: return launch_plane_n<T, 256>(fwd, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

template <> bool has_plane<float>(int N) { return N == 64 || N == 128 || N == 256; }
// N = 64: 0.0246 vs 0.0343 ms per solve.  N = 128 (0.068 vs 0.065) and N = 256
// (0.506 vs 0.463): the plane passes are latency bound (one cluster barrier
// per plane, 8 waves of 36 clusters at N = 256) and lose although W1 no
// longer reaches HBM; they stay available for the A/B (FSP_PLANE=1).
template <> bool plane_default<float>(int N) { return N == 64; }
template <> cudaError_t plane_fwd<float>(int N, const PlaneArgs &a, cudaStream_t s) {
    return launch_plane<float>(true, N, a, s);
}
template <> cudaError_t plane_inv<float>(int N, const PlaneArgs &a, cudaStream_t s) {
    return launch_plane<float>(false, N, a, s);
}

}  // namespace fast
}  // namespace fsp
