// The float flux kernel (flux_kernel.cuh) compiled for 5 and 6 resident
// CTAs of 128 threads per SM (at most 96 and 80 registers per thread, with
// spills), the launch-bounds variants the autotuner times against the
// default of 4 CTAs (128 registers).  A translation unit of its own so that
// the variants compile in parallel with fluxes.cu.
#include "flux_kernel.cuh"

namespace hyd {

namespace {

template <int MINB>
cudaError_t launch_minb(const FluxArgs &a, const float *rec, int riem, int scheme, bool defer,
                        stream_t st) {
    constexpr int E = HYDRO_RIEMANN_EXACT, H = HYDRO_RIEMANN_HLLC;
    if (defer) {
        if (scheme == HYDRO_MFM) return launch_k_fluxes<float, E, HYDRO_MFM, true, MINB>(a, rec, st);
        return launch_k_fluxes<float, E, HYDRO_MFV, true, MINB>(a, rec, st);
    }
    if (riem == H) {
        if (scheme == HYDRO_MFM) return launch_k_fluxes<float, H, HYDRO_MFM, false, MINB>(a, rec, st);
        return launch_k_fluxes<float, H, HYDRO_MFV, false, MINB>(a, rec, st);
    }
    if (scheme == HYDRO_MFM) return launch_k_fluxes<float, E, HYDRO_MFM, false, MINB>(a, rec, st);
    return launch_k_fluxes<float, E, HYDRO_MFV, false, MINB>(a, rec, st);
}

}  // namespace

cudaError_t launch_fluxes_occ(int minb, const FluxArgs &a, const float *rec, int riem, int scheme,
                              bool defer, stream_t st) {
    if (minb == 5) return launch_minb<5>(a, rec, riem, scheme, defer, st);
    if (minb == 6) return launch_minb<6>(a, rec, riem, scheme, defer, st);
    return cudaErrorInvalidValue;
}

}  // namespace hyd
