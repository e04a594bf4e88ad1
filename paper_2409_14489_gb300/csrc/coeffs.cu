// coeffs.cu -- analytic CB-ESSFM coefficients (Sec. II-D), computed on the GPU in FP64.
//
// c_d[m] = (1 / R'^2) double integral over mu, nu in [f_d - R'/2, f_d + R'/2] of
//          K(mu, nu) exp(j 2 pi (mu - nu) m / R')          (Eq. ESSFM_coefficients_general, P = 1)
// for every subband separation f_d = d R' (d = l - i in [-(N_sb - 1), N_sb - 1]) and tap
// m in [-N_c, N_c], with the closed-form kernel of Eq. (kernel_analytic)
//   K = gamma exp(-a L_sp) sinh((a + j b) L_sp) sin(b L) / ((a + j b) sin(b L_sp)),
//   a = alpha / 2, b = 2 pi^2 beta2 nu (mu - nu), L_sp = L / N_sp.
// The double integral is an M x M midpoint rule (the paper's "diagonal of the two-dimensional
// FFT of the kernel on a grid"): c_d[m] = (1/M^2) sum_{p,q} K(mu_p, nu_q) exp(j 2 pi (p - q) m / M).
// One CTA per (d, m) sums the grid with an FP64 block reduction.  The host then assembles the
// DBP taps: w[s][i][l][m + N_c] = P_s Re c_{l-i}[m] (x 3/2 for l != i, Eq. NLPR-multiband-2pol).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "abi_guard.h"
#include "internal.h"
#include "trace.h"

namespace cbessfm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kCoeffThreads = 256;

// K(mu, nu) of Eq. (kernel_analytic) with the limits at b -> 0 and a + j b -> 0.
__device__ double2 kernel_closed_form(double mu, double nu, double beta2, double gamma,
                                      double alpha, double L, int n_spans) {
    const double Lsp = L / n_spans;
    const double a = 0.5 * alpha;
    const double b = 2.0 * kPi * kPi * beta2 * nu * (mu - nu);
    const double xr = a * Lsp, xi = b * Lsp;
    double sr, si;                                    // sinh(x) / x
    if (xr * xr + xi * xi < 1e-16) {
        sr = 1.0 + (xr * xr - xi * xi) / 6.0;
        si = (2.0 * xr * xi) / 6.0;
    } else {
        double sn, cs;
        sincos(xi, &sn, &cs);
        const double hr = sinh(xr) * cs, hi = cosh(xr) * sn;      // sinh(xr + j xi)
        const double den = xr * xr + xi * xi;
        sr = (hr * xr + hi * xi) / den;
        si = (hi * xr - hr * xi) / den;
    }
    const double s_span = sin(b * Lsp);
    double ratio;
    if (fabs(s_span) < 1e-12) {
        // sin(N y) / sin(y) -> N (-1)^(k (N - 1)) at y = k pi
        const double k = rint(b * Lsp / kPi);
        const long long par = ((long long)k * (n_spans - 1)) & 1LL;
        ratio = par ? -(double)n_spans : (double)n_spans;
    } else {
        ratio = sin(b * L) / s_span;
    }
    const double scale = gamma * exp(-a * Lsp) * Lsp * ratio;
    return make_double2(scale * sr, scale * si);
}

// c[d][m]: blockIdx.x = (d + n_sb - 1) * ntaps + (m + nc)
__global__ void coeff_kernel(double2* __restrict__ out, int n_sb, int ntaps, int grid, double rate_sub,
                             double beta2, double gamma, double alpha, double L, int n_spans) {
    __shared__ double red_r[kCoeffThreads], red_i[kCoeffThreads];
    const int nc = (ntaps - 1) / 2;
    const int d = (int)blockIdx.x / ntaps - (n_sb - 1);
    const int m = (int)blockIdx.x % ntaps - nc;
    const double f0 = d * rate_sub - 0.5 * rate_sub;
    const double df = rate_sub / grid;
    double accr = 0.0, acci = 0.0;
    const long long total = (long long)grid * grid;
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int p = (int)(idx / grid), q = (int)(idx - (long long)p * grid);
        const double2 K = kernel_closed_form(f0 + (p + 0.5) * df, f0 + (q + 0.5) * df, beta2, gamma,
                                             alpha, L, n_spans);
        // exp(j 2 pi (p - q) m / M) with the exponent reduced exactly modulo M
        long long r = ((long long)(p - q) * m) % grid;
        if (r < 0) r += grid;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)grid, &sn, &cs);
        accr += K.x * cs - K.y * sn;
        acci += K.x * sn + K.y * cs;
    }
    red_r[threadIdx.x] = accr;
    red_i[threadIdx.x] = acci;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red_r[threadIdx.x] += red_r[threadIdx.x + w];
            red_i[threadIdx.x] += red_i[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double inv = 1.0 / ((double)grid * (double)grid);
        out[blockIdx.x] = make_double2(red_r[0] * inv, red_i[0] * inv);
    }
}

}  // namespace
}  // namespace cbessfm

using namespace cbessfm;

extern "C" {

static cbessfm_status analytic_taps_body(const cbessfm_link* link, int bands, int steps,
                                         int spans_per_step, const double* step_power, int ntaps,
                                         int grid, double* taps, double* response) {
    if (link == nullptr || taps == nullptr || (steps > 0 && step_power == nullptr))
        return fail(CBESSFM_ERR_INVALID_ARG, "link, taps or step_power is NULL");
    if (bands < 1 || bands > 16) return fail(CBESSFM_ERR_INVALID_ARG, "bands must be in [1, 16]");
    if (steps < 1 || steps > 4096) return fail(CBESSFM_ERR_INVALID_ARG, "steps must be in [1, 4096]");
    if (ntaps < 1 || (ntaps & 1) == 0 || ntaps > 1023)
        return fail(CBESSFM_ERR_INVALID_ARG, "ntaps must be odd and in [1, 1023]");
    if (grid < ntaps || grid > 4096)
        return fail(CBESSFM_ERR_INVALID_ARG, "grid must be in [ntaps, 4096]");
    if (spans_per_step < 1) return fail(CBESSFM_ERR_INVALID_ARG, "spans_per_step must be >= 1");
    if (!(link->sample_rate > 0.0) || !(link->span_length > 0.0) || link->n_spans < 1)
        return fail(CBESSFM_ERR_INVALID_ARG, "link sample_rate, span_length, n_spans must be positive");
    if (!std::isfinite(link->beta2) || !std::isfinite(link->gamma) || !(link->alpha >= 0.0))
        return fail(CBESSFM_ERR_INVALID_ARG, "beta2, gamma must be finite and alpha >= 0");
    const double L = link->span_length * link->n_spans / steps;
    if (spans_per_step > 1 && (long long)steps * spans_per_step != link->n_spans)
        return fail(CBESSFM_ERR_INVALID_ARG,
                    "spans_per_step > 1 needs steps * spans_per_step == n_spans (%d * %d != %d)",
                    steps, spans_per_step, link->n_spans);
    const int n_sep = 2 * bands - 1;
    const int n_out = n_sep * ntaps;
    std::vector<double2> c(n_out);                 // before the device allocation (abi_guard.h)
    double2* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_out, sizeof(double2) * n_out);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(coefficients)");
    coeff_kernel<<<n_out, kCoeffThreads>>>(d_out, bands, ntaps, grid, link->sample_rate / bands,
                                           link->beta2, link->gamma, link->alpha, L, spans_per_step);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(c.data(), d_out, sizeof(double2) * n_out, cudaMemcpyDeviceToHost);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(e, "analytic coefficients");
    for (int s = 0; s < steps; ++s)
        for (int i = 0; i < bands; ++i)
            for (int l = 0; l < bands; ++l)
                for (int m = 0; m < ntaps; ++m) {
                    const double re = c[(size_t)(l - i + bands - 1) * ntaps + m].x;
                    taps[(((size_t)s * bands + i) * bands + l) * ntaps + m] =
                        step_power[s] * re * (i == l ? 1.0 : 1.5);
                }
    if (response != nullptr)
        for (int k = 0; k < n_out; ++k) {
            response[2 * k] = c[k].x;
            response[2 * k + 1] = c[k].y;
        }
    return CBESSFM_OK;
}

cbessfm_status cbessfm_analytic_taps(const cbessfm_link* link, int bands, int steps,
                                     int spans_per_step, const double* step_power, int ntaps,
                                     int grid, double* taps, double* response) {
    TraceRange trace_range("cbessfm:analytic_taps");
    clear_error();
    return abi_guard([&] {
        return analytic_taps_body(link, bands, steps, spans_per_step, step_power, ntaps, grid,
                                  taps, response);
    });
}

}  // extern "C"
