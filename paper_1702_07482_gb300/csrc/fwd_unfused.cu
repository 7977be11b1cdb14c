// Launcher of the unfused three-kernel baseline stage.
#include "launch.h"
#include "unfused.cuh"

namespace tnrd {

namespace {

template <int KS>
cudaError_t launch_ks(const UnfArgs& a, int N, cudaStream_t s)
{
    const int npix = a.H * a.W;
    const dim3 g1((npix + 255) / 256, a.nfilt, N);
    unf_bank_phi<KS><<<g1, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 g2((npix + 255) / 256, N);
    const size_t smem = sizeof(float) * (size_t)a.nfilt * KS * KS;
    unf_adjoint<KS><<<g2, 256, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unf_prox<<<g2, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_unfused_fwd(int ks, const UnfArgs& a, int N, cudaStream_t s)
{
    switch (ks) {
    case 3: return launch_ks<3>(a, N, s);
    case 5: return launch_ks<5>(a, N, s);
    case 7: return launch_ks<7>(a, N, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnrd
