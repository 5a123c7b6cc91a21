// kt_advect.cu -- stoichiometry-compatible species advection (Sec. 2.1.3 of the paper):
// one directional sweep of piecewise-linear reconstruction with the slope corrections
// projected onto the null space of the element matrix, upwind species fluxes
// F^s = x^s F^rho (Eq. method-flux-sp) and the conservative update, fused in one pass.
//
// The correction of a cell at its two interfaces is chi = +-dx/2 s (s: the limited
// slopes of x^s = n^s/rho), so projecting chi onto the stoichiometric space S = null(N)
// is projecting s once: s' = s - V_r (V_r^T s), with V_r an orthonormal basis of N's row
// space (rank <= 8).  That costs O(N_species N_elements) per cell instead of a dense
// N_species^2 product, and leaves N s' = 0 exactly up to rounding.
//
// Layout: lines of L cells, periodic; n[s][line][j] (species-major SoA), rho and the mass
// flux [line][j] (mass_flux[j] at the interface j-1/2).  A block owns a segment of B
// cells of one line and stages x^s = n^s/rho for the segment plus two cells each side in
// shared memory (coalesced along j); its threads then form the projected slopes of B+2
// cells, the fluxes at the B+1 interfaces and the B updates.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kt_internal.h"

namespace kt {
namespace {

constexpr int kAdvMaxRank = kMaxElements;

struct AdvArgs {
    long long nlines, L;
    int ns, rank, B, project;
    const double *n_in, *rho, *mflux, *n_base;
    double *n_out;
    double dx, dtdx, alpha;
    double vr[kAdvMaxRank * 256];   // V_r [ns][rank] (ns <= 256)
};

// slope of the modified van Leer limiter: sgn(a) min(2|a||b|/(|a|+|b|), |b|), zero at
// extrema (a b <= 0); the uniform-grid geometric factor 2c/(c+d) is 1
__device__ __forceinline__ double vl_slope(double a, double b)
{
    if (!(a * b > 0.0)) return 0.0;
    const double aa = fabs(a), bb = fabs(b);
    double phi = 2.0 * aa / (aa + bb);
    if (phi > 1.0) phi = 1.0;
    return copysign(phi * bb, a);
}

__global__ void advect_kernel(const AdvArgs *__restrict__ p)
{
    extern __shared__ double sm[];
    const int ns = p->ns, B = p->B, W = B + 4;
    const long long L = p->L;
    const long long line = blockIdx.y;
    const long long j0 = static_cast<long long>(blockIdx.x) * B;
    double *X = sm;                         // [ns][B+4]: x at cells j0-2 .. j0+B+1
    double *S = X + ns * W;                 // [ns][B+2]: projected slopes, cells j0-1 .. j0+B
    double *F = S + ns * (B + 2);           // [ns][B+1]: fluxes at j0-1/2 .. j0+B-1/2
    const double *rho = p->rho + line * L;
    const double *mf = p->mflux + line * L;
    auto wrap = [&](long long j) { j %= L; return j < 0 ? j + L : j; };

    // stage x = n / rho (periodic halo)
    for (int q = threadIdx.x; q < W; q += blockDim.x) {
        const long long j = wrap(j0 - 2 + q);
        const double inv = 1.0 / rho[j];
        for (int s = 0; s < ns; ++s) X[s * W + q] = p->n_in[(s * p->nlines + line) * L + j] * inv;
    }
    __syncthreads();
    // projected slopes of cells j0-1 .. j0+B (index c = 0 .. B+1, X index c+1)
    const double idx = 1.0 / p->dx;
    for (int c = threadIdx.x; c < B + 2; c += blockDim.x) {
        double coef[kAdvMaxRank];
#pragma unroll
        for (int k = 0; k < kAdvMaxRank; ++k) coef[k] = 0.0;
        for (int s = 0; s < ns; ++s) {
            const double *xs = X + s * W + c + 1;
            const double sl = vl_slope((xs[1] - xs[0]) * idx, (xs[0] - xs[-1]) * idx);
            S[s * (B + 2) + c] = sl;
            if (p->project)
                for (int k = 0; k < p->rank; ++k) coef[k] += p->vr[s * p->rank + k] * sl;
        }
        if (p->project) {
            for (int s = 0; s < ns; ++s) {
                double d = 0.0;
                for (int k = 0; k < p->rank; ++k) d += p->vr[s * p->rank + k] * coef[k];
                S[s * (B + 2) + c] -= d;
            }
        }
    }
    __syncthreads();
    // fluxes at the interfaces j-1/2, j = j0 .. j0+B (index i = 0 .. B): left state from
    // cell j-1 (upper side), right state from cell j (lower side), upwind by the mass flux
    const double hdx = 0.5 * p->dx;
    for (int i = threadIdx.x; i < B + 1; i += blockDim.x) {
        const double m = mf[wrap(j0 + i)];
        for (int s = 0; s < ns; ++s) {
            const double xl = X[s * W + i + 1] + hdx * S[s * (B + 2) + i];
            const double xr = X[s * W + i + 2] - hdx * S[s * (B + 2) + i + 1];
            F[s * (B + 1) + i] = (m > 0.0 ? xl : xr) * m;
        }
    }
    __syncthreads();
    // conservative update (and the Runge-Kutta blend with n_base)
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const long long j = j0 + i;
        if (j >= L) break;
        for (int s = 0; s < ns; ++s) {
            const long long g = (s * p->nlines + line) * L + j;
            const double v = p->n_in[g] - p->dtdx * (F[s * (B + 1) + i + 1] - F[s * (B + 1) + i]);
            p->n_out[g] = p->n_base ? p->alpha * p->n_base[g] + (1.0 - p->alpha) * v : v;
        }
    }
}

}  // namespace
}  // namespace kt

extern "C" KT_API int kt_advect_sweep(const kt_network *net, int64_t nlines, int64_t L, const double *n_in,
                                      const double *rho, const double *mass_flux, double dx, double dtdx,
                                      double alpha, const double *n_base, double *n_out, int project,
                                      void *scratch, void *cuda_stream)
{
    using namespace kt;
    int ns = 0, rank = 0;
    double vr[kAdvMaxRank * 256];
    int rc = network_element_basis(net, vr, &ns, &rank);
    if (rc) return rc;
    if (nlines < 0 || L < 0 || !(dx > 0) || !std::isfinite(dtdx) || ns > 256) {
        set_error("kt_advect_sweep: bad sizes or dx");
        return KT_EINVAL;
    }
    if (nlines == 0 || L == 0) return KT_OK;
    if (L < 3) {
        set_error("kt_advect_sweep: a periodic line needs at least 3 cells");
        return KT_EINVAL;
    }
    if (!n_in || !rho || !mass_flux || !n_out || !scratch || nlines > 65535) {
        set_error("kt_advect_sweep: NULL device buffer or more than 65535 lines");
        return KT_EINVAL;
    }
    if (n_out == n_in) {
        set_error("kt_advect_sweep: n_out must not alias n_in (neighbouring blocks read it)");
        return KT_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(scratch) % 16) {
        set_error("kt_advect_sweep: scratch not 16-B aligned");
        return KT_EINVAL;
    }
    // segment length: the staged tile (x, slopes, fluxes) within 96 KB
    int B = 128;
    while (B > 16 && static_cast<size_t>(3 * B + 7) * ns * sizeof(double) > 96 * 1024) B /= 2;
    if (static_cast<size_t>(3 * B + 7) * ns * sizeof(double) > 200 * 1024) {
        set_error("kt_advect_sweep: too many species for the shared-memory tile");
        return KT_EUNSUPPORTED;
    }
    AdvArgs h{};
    h.nlines = nlines;
    h.L = L;
    h.ns = ns;
    h.rank = rank;
    h.B = B;
    h.project = project ? 1 : 0;
    h.n_in = n_in;
    h.rho = rho;
    h.mflux = mass_flux;
    h.n_base = n_base;
    h.n_out = n_out;
    h.dx = dx;
    h.dtdx = dtdx;
    h.alpha = alpha;
    for (int q = 0; q < ns * rank; ++q) h.vr[q] = vr[q];
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    AdvArgs *dev = static_cast<AdvArgs *>(scratch);
    cudaError_t e = cudaMemcpyAsync(dev, &h, sizeof(AdvArgs), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error(cudaGetErrorString(e));
        return KT_ECUDA;
    }
    const size_t smem = static_cast<size_t>(3 * B + 7) * ns * sizeof(double);
    e = cudaFuncSetAttribute(advect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) {
        set_error(cudaGetErrorString(e));
        return KT_ECUDA;
    }
    const dim3 grid(static_cast<unsigned>((L + B - 1) / B), static_cast<unsigned>(nlines));
    advect_kernel<<<grid, B, smem, s>>>(dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(cudaGetErrorString(e));
        return KT_ECUDA;
    }
    return KT_OK;
}

extern "C" KT_API size_t kt_advect_scratch_bytes(void) { return sizeof(kt::AdvArgs); }
