// kt_ray.cu -- ray tracing on a Cartesian mesh with Beer-Lambert deposition (Sec. 3 of
// the paper: Eqs. cart-dl, method-rt-ph-num, method-rad-equiv-flux, method-rt-abs).
//
// One thread per ray.  The ray walks the cells it crosses by incremental face stepping
// (the exit length of a cell is the smallest root of the axis-plane equations of Eq.
// cart-dl; here each axis's next crossing distance is recomputed from the ray origin,
// t_a = (face_a - x0_a)/d_a, so no position error accumulates along the ray).  In each
// cell it deposits, per energy bin, the path-averaged effective flux
// N dl/(dV dt) (1 - e^-tau)/tau and the absorbed photons N (1 - e^-tau), tau = kappa dl,
// into per-cell accumulators (FP64 atomics: rays cross shared cells), and carries
// N e^-tau on.  A walk crosses at most nx + ny + nz cells, which bounds the loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kt_internal.h"

namespace kt {
namespace {

constexpr int kRayMaxBins = 8;

struct RayArgs {
    int nx, ny, nz, nb;
    double hx, hy, hz, dt;
    long long nrays;
    const double *kappa, *org, *dir, *n0;
    double *feff, *absorbed, *escaped;
};

__global__ void ray_kernel(const RayArgs a)
{
    const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= a.nrays) return;
    const double x0[3] = {a.org[3 * q], a.org[3 * q + 1], a.org[3 * q + 2]};
    const double d[3] = {a.dir[3 * q], a.dir[3 * q + 1], a.dir[3 * q + 2]};
    const double h[3] = {a.hx, a.hy, a.hz};
    const int n[3] = {a.nx, a.ny, a.nz};
    double N[kRayMaxBins];
    for (int b = 0; b < a.nb; ++b) N[b] = a.n0[q * a.nb + b];
    int c[3];
    bool inside = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c[k] = static_cast<int>(floor(x0[k] / h[k]));
        inside = inside && c[k] >= 0 && c[k] < n[k] && x0[k] >= 0.0;
    }
    const double dV = a.hx * a.hy * a.hz, inv_dVdt = 1.0 / (dV * a.dt);
    const long long ncell = static_cast<long long>(a.nx) * a.ny * a.nz;
    double t = 0.0;
    const int max_steps = a.nx + a.ny + a.nz + 3;
    for (int it = 0; inside && it < max_steps; ++it) {
        // next face crossing of each axis, from the origin
        double tn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (d[k] > 0.0) tn[k] = ((c[k] + 1) * h[k] - x0[k]) / d[k];
            else if (d[k] < 0.0) tn[k] = (c[k] * h[k] - x0[k]) / d[k];
            else tn[k] = INFINITY;
        }
        int ax = 0;
        if (tn[1] < tn[ax]) ax = 1;
        if (tn[2] < tn[ax]) ax = 2;
        double dl = tn[ax] - t;
        if (dl < 0.0) dl = 0.0;
        const long long cell = (static_cast<long long>(c[0]) * a.ny + c[1]) * a.nz + c[2];
        for (int b = 0; b < a.nb; ++b) {
            const double tau = a.kappa[b * ncell + cell] * dl;
            const double att = exp(-tau);
            const double phi = tau > 0.0 ? -expm1(-tau) / tau : 1.0;
            atomicAdd(&a.feff[b * ncell + cell], N[b] * dl * inv_dVdt * phi);
            atomicAdd(&a.absorbed[b * ncell + cell], N[b] * (1.0 - att));
            N[b] *= att;
        }
        t = tn[ax];
        c[ax] += d[ax] > 0.0 ? 1 : -1;
        inside = c[ax] >= 0 && c[ax] < n[ax];
    }
    if (a.escaped)
        for (int b = 0; b < a.nb; ++b) a.escaped[q * a.nb + b] = N[b];
}

// Isotropic point source: Fibonacci-lattice directions (z_k = 1 - (2k+1)/n, azimuth
// k times the golden angle), solid angle 4 pi / n each, N = L dOmega/(4 pi) dt per bin.
constexpr double kPi = 3.141592653589793;

__device__ __forceinline__ void point_source_ray(long long k, double sx, double sy, double sz,
                                                 const double *lum_dt_over_n, int nb, long long nrays, double *org,
                                                 double *dir, double *n0)
{
    const double golden = kPi * (3.0 - sqrt(5.0));
    const double z = 1.0 - (2.0 * static_cast<double>(k) + 1.0) / static_cast<double>(nrays);
    const double r = sqrt(fmax(0.0, 1.0 - z * z));
    const double ph = static_cast<double>(k) * golden;
    double s, c;
    sincos(ph, &s, &c);
    org[3 * k] = sx;
    org[3 * k + 1] = sy;
    org[3 * k + 2] = sz;
    dir[3 * k] = r * c;
    dir[3 * k + 1] = r * s;
    dir[3 * k + 2] = z;
    for (int b = 0; b < nb; ++b) n0[k * nb + b] = lum_dt_over_n[b];
}

struct LumArg {
    double v[kRayMaxBins];
};

__global__ void point_source_kernel(double sx, double sy, double sz, const LumArg lum, int nb, long long nrays,
                                    double *org, double *dir, double *n0)
{
    const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < nrays) point_source_ray(k, sx, sy, sz, lum.v, nb, nrays, org, dir, n0);
}

}  // namespace
}  // namespace kt

extern "C" KT_API int kt_raytrace(int nx, int ny, int nz, double hx, double hy, double hz, int nbins,
                                  const double *kappa, int64_t nrays, const double *origins,
                                  const double *dirs, const double *n0, double dt, double *feff,
                                  double *absorbed, double *escaped, void *cuda_stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || !(hx > 0) || !(hy > 0) || !(hz > 0) || nbins < 1 ||
        nbins > kt::kRayMaxBins || nrays < 0 || !(dt > 0)) {
        kt::set_error("kt_raytrace: bad grid, bins, ray count or dt");
        return KT_EINVAL;
    }
    if (nrays == 0) return KT_OK;
    if (!kappa || !origins || !dirs || !n0 || !feff || !absorbed) {
        kt::set_error("kt_raytrace: NULL device buffer");
        return KT_EINVAL;
    }
    kt::RayArgs a{nx, ny, nz, nbins, hx, hy, hz, dt, nrays, kappa, origins, dirs, n0, feff, absorbed, escaped};
    const int threads = 128;
    kt::ray_kernel<<<static_cast<unsigned>((nrays + threads - 1) / threads), threads, 0,
                     static_cast<cudaStream_t>(cuda_stream)>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        kt::set_error(cudaGetErrorString(e));
        return KT_ECUDA;
    }
    return KT_OK;
}

extern "C" KT_API int kt_rays_point_source(const double *src, const double *lum, int nbins, double dt,
                                           int64_t nrays, double *origins, double *dirs, double *n0,
                                           void *cuda_stream)
{
    if (!src || !lum || nbins < 1 || nbins > kt::kRayMaxBins || nrays < 1 || !(dt > 0) || !origins || !dirs ||
        !n0) {
        kt::set_error("kt_rays_point_source: bad argument");
        return KT_EINVAL;
    }
    kt::LumArg l{};
    for (int b = 0; b < nbins; ++b) l.v[b] = lum[b] * dt / static_cast<double>(nrays);
    const int threads = 128;
    kt::point_source_kernel<<<static_cast<unsigned>((nrays + threads - 1) / threads), threads, 0,
                                static_cast<cudaStream_t>(cuda_stream)>>>(src[0], src[1], src[2], l, nbins, nrays,
                                                                          origins, dirs, n0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        kt::set_error(cudaGetErrorString(e));
        return KT_ECUDA;
    }
    return KT_OK;
}
