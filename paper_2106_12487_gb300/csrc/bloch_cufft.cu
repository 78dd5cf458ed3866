// Plain-form baseline of the stiffness operator (fft_variant 2): Eq. (hatA)
// evaluated literally with library 3D FFTs (cuFFT) and three unfused pointwise
// kernels.  This is the reference point the fused passes are measured
// against; it is not used by the default path.
//   gamma = sym(q (x) U) (Fourier, 6 comps) -> F^-1 (cuFFT, 6 comps)
//   sigma = C_g(x) gamma / V (real space)    -> F   (cuFFT, 6 comps)
//   out_i = q_j sigma_ij (Fourier)
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <map>
#include <type_traits>
#include <string>
#include <utility>

#include "internal.h"

namespace bloch {

template <typename T>
__global__ void k_strain6(const cplx_t<T>* __restrict__ U, cplx_t<T>* __restrict__ E, const T* __restrict__ qtab,
                          Geo g) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const C* u = U + (size_t)b * 3 * g.V;
    C* e = E + (size_t)b * 6 * g.V;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        T qx, qy, qz;
        voxel_q(qb, g, v, qx, qy, qz);
        const C ux = u[v], uy = u[g.V + v], uz = u[2 * g.V + v];
        e[v] = cscale(ux, qx);
        e[g.V + v] = cscale(uy, qy);
        e[2 * g.V + v] = cscale(uz, qz);
        e[3 * g.V + v] = cadd(cscale(uy, qz), cscale(uz, qy));
        e[4 * g.V + v] = cadd(cscale(ux, qz), cscale(uz, qx));
        e[5 * g.V + v] = cadd(cscale(ux, qy), cscale(uy, qx));
    }
}

template <typename T>
__global__ void k_stress6(cplx_t<T>* E, const int32_t* __restrict__ ids, const T* __restrict__ Ctab, Geo g) {
    using C = cplx_t<T>;
    C* e = E + (size_t)blockIdx.y * 6 * g.V;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        const T* Cg = Ctab + (size_t)ids[v] * 36;
        C gam[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) gam[c] = e[(size_t)c * g.V + v];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            T sr = 0, si = 0;
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const T cij = __ldg(Cg + i * 6 + j);
                sr = fma(cij, gam[j].x, sr);
                si = fma(cij, gam[j].y, si);
            }
            e[(size_t)i * g.V + v] = mk(sr, si);
        }
    }
}

template <typename T>
__global__ void k_div3(const cplx_t<T>* __restrict__ E, cplx_t<T>* __restrict__ out, const T* __restrict__ qtab,
                       Geo g, T scale) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const C* e = E + (size_t)b * 6 * g.V;
    C* o = out + (size_t)b * 3 * g.V;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        T qx, qy, qz;
        voxel_q(qb, g, v, qx, qy, qz);
        const C s11 = e[v], s22 = e[g.V + v], s33 = e[2 * g.V + v];
        const C s23 = e[3 * g.V + v], s13 = e[4 * g.V + v], s12 = e[5 * g.V + v];
        o[v] = cscale(cadd(cadd(cscale(s11, qx), cscale(s12, qy)), cscale(s13, qz)), scale);
        o[g.V + v] = cscale(cadd(cadd(cscale(s12, qx), cscale(s22, qy)), cscale(s23, qz)), scale);
        o[2 * g.V + v] = cscale(cadd(cadd(cscale(s13, qx), cscale(s23, qy)), cscale(s33, qz)), scale);
    }
}

// cuFFT plans keyed by (plan, precision, transforms per call)
static std::map<std::pair<const bloch_plan*, int>, cufftHandle> g_plans;

static cufftHandle get_plan(bloch_plan* pl, bool fp64, int batch) {
    const auto key = std::make_pair((const bloch_plan*)pl, (fp64 ? 1 : 0) | (batch << 1));
    auto it = g_plans.find(key);
    if (it != g_plans.end()) return it->second;
    cufftHandle h = 0;
    int n[3] = {pl->Nz, pl->Ny, pl->Nx};
    if (cufftPlanMany(&h, 3, n, nullptr, 1, (int)pl->V, nullptr, 1, (int)pl->V, fp64 ? CUFFT_Z2Z : CUFFT_C2C,
                      batch) != CUFFT_SUCCESS)
        return 0;
    cufftSetStream(h, pl->stream);
    g_plans[key] = h;
    return h;
}

void cufft_release(const bloch_plan* pl) {
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (it->first.first == pl) {
            cufftDestroy(it->second);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

template <typename T>
bool cufft_launch_K(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale, cplx_t<T>* E,
                    const T* qtab, const T* Ctab, const Geo& g) {
    constexpr bool fp64 = std::is_same<T, double>::value;
    cufftHandle h = get_plan(pl, fp64, 6 * nb);
    if (!h) return false;
    const int blocks = (int)std::min<long long>((pl->V + 255) / 256, 2048);
    dim3 gr(blocks, nb);
    pl->launches += 3;
    k_strain6<T><<<gr, 256, 0, pl->stream>>>(u, E, qtab, g);
    if constexpr (fp64) {
        if (cufftExecZ2Z(h, (cufftDoubleComplex*)E, (cufftDoubleComplex*)E, CUFFT_INVERSE) != CUFFT_SUCCESS)
            return false;
    } else {
        if (cufftExecC2C(h, (cufftComplex*)E, (cufftComplex*)E, CUFFT_INVERSE) != CUFFT_SUCCESS) return false;
    }
    k_stress6<T><<<gr, 256, 0, pl->stream>>>(E, pl->d_ids, Ctab, g);
    if constexpr (fp64) {
        if (cufftExecZ2Z(h, (cufftDoubleComplex*)E, (cufftDoubleComplex*)E, CUFFT_FORWARD) != CUFFT_SUCCESS)
            return false;
    } else {
        if (cufftExecC2C(h, (cufftComplex*)E, (cufftComplex*)E, CUFFT_FORWARD) != CUFFT_SUCCESS) return false;
    }
    k_div3<T><<<gr, 256, 0, pl->stream>>>(E, out, qtab, g, out_scale);
    return true;
}

template bool cufft_launch_K<float>(bloch_plan*, int, const float2*, float2*, float, float2*, const float*,
                                    const float*, const Geo&);
template bool cufft_launch_K<double>(bloch_plan*, int, const double2*, double2*, double, double2*, const double*,
                                     const double*, const Geo&);

}  // namespace bloch
