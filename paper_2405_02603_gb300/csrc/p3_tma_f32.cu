// p3_tma_f32.cu -- host launcher of the TMA-staged persistent P3
// (p3_tma.cuh), single precision, lines of 2N = 128, 256, 512.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "p3_tma.cuh"

namespace fsp {
namespace fast {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// W2[z][k_y][k_x] (z < N, k_y < 2N, row pitch P complex) as a 3D tensor of
// 4-byte elements; box = L lines x 1 k_y row x N positions.
template <typename T> bool encode_w2(CUtensorMap &m, void *w2, int N, int P, int L) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    constexpr int XE = (int)(sizeof(cx_t<T>) / 4);
    const cuuint64_t dims[3] = {(cuuint64_t)P * XE, (cuuint64_t)2 * N, (cuuint64_t)N};
    const cuuint64_t strides[2] = {(cuuint64_t)P * sizeof(cx_t<T>), (cuuint64_t)2 * N * P * sizeof(cx_t<T>)};
    const cuuint32_t box[3] = {(cuuint32_t)(L * XE), 1u, (cuuint32_t)N};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, w2, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int n>
cudaError_t launch_p3_tma_n(void *w2, const void *S, const void *tw, const P3Wait &w, cudaStream_t s) {
    using K = ColCfg<T, n, COL_FMI>;
    constexpr int N = n / 2, L = K::L, NTH = L * (n / K::V);
    static_assert(N % L == 0, "tiles must cover k_x < N exactly");
    const char *tv = std::getenv("FSP_P3_TWS");
    const bool tws = tv ? tv[0] == '1' : ColOpt<T, COL_FMI, n>::TWS;
    auto kern = tws ? k_p3_tma<T, n, K::V, L, K::R1, K::R2, K::R3, true> : k_p3_tma<T, n, K::V, L, K::R1, K::R2, K::R3, false>;
    const size_t sm = tws ? p3_tma_smem<T, n, L, true>() : p3_tma_smem<T, n, L, false>();
    // a box starts 16-byte aligned: the workspace base is, and every row and
    // tile offset is a multiple of 128 bytes (pitch and L multiples of 16)
    if ((reinterpret_cast<uintptr_t>(w2) & 15u) != 0) return cudaErrorInvalidValue;
    CUtensorMap m;
    if (!encode_w2<T>(m, w2, N, row_pitch(N), L)) return cudaErrorInvalidValue;
    cudaError_t e;
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTH, sm)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    P3TmaArgs a{};
    a.w2 = w2, a.S = S, a.tw = tw, a.err = w.err;
    a.timeout_ns = w.timeout_ns, a.extra_tx = w.extra_tx;
    a.ntiles_nyq = 2 * N / L;
    a.ntiles = a.ntiles_nyq + 2 * N * (N / L);
    // every CTA takes one Nyquist tile at most (they are the slow ones)
    const int grid = std::min(a.ntiles, std::max(per_sm * sms, a.ntiles_nyq));
    kern<<<grid, NTH, sm, s>>>(m, a);
    return cudaGetLastError();
}

}  // namespace

template <> bool has_p3_tma<float>(int N) { return N == 64 || N == 128 || N == 256; }

template <> cudaError_t p3_tma<float>(int N, void *w2, const void *S, const void *tw, const P3Wait &w, cudaStream_t s) {
    switch (N) {
    case 64: return launch_p3_tma_n<float, 128>(w2, S, tw, w, s);
    case 128: return launch_p3_tma_n<float, 256>(w2, S, tw, w, s);
    case 256: return launch_p3_tma_n<float, 512>(w2, S, tw, w, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fast
}  // namespace fsp
