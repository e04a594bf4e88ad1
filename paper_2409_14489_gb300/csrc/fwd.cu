// fwd.cu -- FP64 GVD table builder and dispatch of the forward chain kernel instantiations.
#include "device_common.cuh"
#include "internal.h"
#include "storage_convert.h"
#include "fwd_launch.h"

namespace cbessfm {

// ------------------------------------------------------------------------------------------
// FP64 table builder: GVD factors of the three step kinds for every subband bin
// ------------------------------------------------------------------------------------------
// The forward chain reads the same factors from a half table indexed by |b| (the factor depends
// on f^2 only): gvd_half[kind][m] = h(m R / N), m = 0 .. N/2, for the three kinds, plus a fourth
// kind, no dispersion with the 1/N scale, that opens the later passes of the streamed form.
__global__ void build_gvd_half_kernel(float2* __restrict__ half, long long N, double beta2,
                                      double rate, double dz0, double dz1, double dz2,
                                      double scale0, double scale12) {
    const long long per = N / 2 + 1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * per) return;
    const int tbl = (int)(idx / per);
    if (tbl == 3) {
        half[idx] = make_float2((float)scale0, 0.0f);
        return;
    }
    const long long m = idx - tbl * per;
    const double f = (double)m * rate / (double)N;
    const double dz = tbl == 0 ? dz0 : (tbl == 1 ? dz1 : dz2);
    const double turns = 3.14159265358979323846 * beta2 * dz * f * f;
    const double frac = turns - floor(turns);
    double sn, cs;
    sincospi(2.0 * frac, &sn, &cs);
    const double sc = tbl == 0 ? scale0 : scale12;
    half[idx] = make_float2((float)(cs * sc), (float)(sn * sc));
}

__global__ void build_gvd_kernel(float2* __restrict__ gvd, int n_sb, int np, double beta2,
                                 double rate, double dz0, double dz1, double dz2, double scale0,
                                 double scale12) {
    const int per = n_sb * np;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * per) return;
    const int tbl = idx / per;
    const int r = idx - tbl * per;
    const int i = r / np;
    const int kap = r - i * np;
    const long long N = (long long)n_sb * np;
    const long long b = -N / 2 + (long long)i * np + np / 2 + (kap < np / 2 ? kap : kap - np);
    const double f = (double)b * rate / (double)N;
    const double dz = tbl == 0 ? dz0 : (tbl == 1 ? dz1 : dz2);
    // phase / (2 pi) = pi beta2 dz f^2, reduced to [0, 1) turns before the sine and cosine
    const double turns = 3.14159265358979323846 * beta2 * dz * f * f;
    const double frac = turns - floor(turns);
    double sn, cs;
    sincospi(2.0 * frac, &sn, &cs);
    const double sc = tbl == 0 ? scale0 : scale12;
    gvd[idx] = make_float2((float)(cs * sc), (float)(sn * sc));
}

cudaError_t launch_build_gvd(const PlanImpl& p, cudaStream_t stream) {
    const int np = p.n_fft;
    const double Ls = p.step_length;
    double dz0, dz1, dz2;
    if (p.n_st == 0) {
        dz0 = p.link.span_length * p.link.n_spans;
        dz1 = dz2 = 0.0;
    } else {
        dz0 = (1.0 - p.ratio) * Ls;
        dz1 = Ls;
        dz2 = p.ratio * Ls;
    }
    const int total = 3 * p.n_sb * np;
    build_gvd_kernel<<<(total + 255) / 256, 256, 0, stream>>>(
        p.d_gvd, p.n_sb, np, p.link.beta2, p.link.sample_rate, dz0, dz1, dz2, 1.0 / (double)p.N,
        1.0 / (double)np);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long half = 4LL * (p.N / 2 + 1);
    build_gvd_half_kernel<<<(unsigned)((half + 255) / 256), 256, 0, stream>>>(
        p.d_gvd_half, p.N, p.link.beta2, p.link.sample_rate, dz0, dz1, dz2, 1.0 / (double)p.N,
        1.0 / (double)np);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
template <int ST>
static cudaError_t prepare_st(int np, int smem_bytes) {
    switch (np) {
        case 16: return fwd_prepare<16, ST>(smem_bytes);
        case 32: return fwd_prepare<32, ST>(smem_bytes);
        case 64: return fwd_prepare<64, ST>(smem_bytes);
        case 128: return fwd_prepare<128, ST>(smem_bytes);
        case 256: return fwd_prepare<256, ST>(smem_bytes);
        case 512: return fwd_prepare<512, ST>(smem_bytes);
        case 1024: return fwd_prepare<1024, ST>(smem_bytes);
        case 2048: return fwd_prepare<2048, ST>(smem_bytes);
        default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t launch_st(int np, const ChainArgs& a, int threads, cudaStream_t stream) {
    switch (np) {
        case 16: return fwd_launch<16, ST>(a, threads, stream);
        case 32: return fwd_launch<32, ST>(a, threads, stream);
        case 64: return fwd_launch<64, ST>(a, threads, stream);
        case 128: return fwd_launch<128, ST>(a, threads, stream);
        case 256: return fwd_launch<256, ST>(a, threads, stream);
        case 512: return fwd_launch<512, ST>(a, threads, stream);
        case 1024: return fwd_launch<1024, ST>(a, threads, stream);
        case 2048: return fwd_launch<2048, ST>(a, threads, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int ST>
static cudaError_t persistent_st(int np, const ChainArgs* jobs, const int2* items, int n_items,
                                 unsigned int* counter, int n_sb, int G, int region_bytes,
                                 int tbl_bytes, int per_pol, int threads, int grid,
                                 cudaStream_t stream) {
#define CB_CASE(NP)                                                                              \
    case NP:                                                                                     \
        return fwd_persistent_launch<NP, ST>(jobs, items, n_items, counter, n_sb, G, region_bytes, \
                                             tbl_bytes, per_pol, threads, grid, stream);
    switch (np) {
        CB_CASE(16) CB_CASE(32) CB_CASE(64) CB_CASE(128) CB_CASE(256) CB_CASE(512) CB_CASE(1024)
        CB_CASE(2048)
        default: return cudaErrorInvalidValue;
    }
#undef CB_CASE
}

template <int ST>
static cudaError_t occupancy_st(int np, int threads, int smem_bytes, int* ctas) {
#define CB_CASE(NP) \
    case NP: return fwd_persistent_occupancy<NP, ST>(threads, smem_bytes, ctas);
    switch (np) {
        CB_CASE(16) CB_CASE(32) CB_CASE(64) CB_CASE(128) CB_CASE(256) CB_CASE(512) CB_CASE(1024)
        CB_CASE(2048)
        default: return cudaErrorInvalidValue;
    }
#undef CB_CASE
}

cudaError_t launch_forward_persistent(int np, int storage, const ChainArgs* jobs, const int2* items,
                                      int n_items, unsigned int* counter, int n_sb, int G,
                                      int region_bytes, int tbl_bytes, int per_pol, int threads,
                                      int grid, cudaStream_t stream) {
    switch (storage) {
        case 0: return persistent_st<0>(np, jobs, items, n_items, counter, n_sb, G, region_bytes, tbl_bytes, per_pol, threads, grid, stream);
        case 1: return persistent_st<1>(np, jobs, items, n_items, counter, n_sb, G, region_bytes, tbl_bytes, per_pol, threads, grid, stream);
        case 2: return persistent_st<2>(np, jobs, items, n_items, counter, n_sb, G, region_bytes, tbl_bytes, per_pol, threads, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t forward_persistent_occupancy(int np, int storage, int threads, int smem_bytes,
                                         int* ctas_per_sm) {
    switch (storage) {
        case 0: return occupancy_st<0>(np, threads, smem_bytes, ctas_per_sm);
        case 1: return occupancy_st<1>(np, threads, smem_bytes, ctas_per_sm);
        case 2: return occupancy_st<2>(np, threads, smem_bytes, ctas_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_forward(int np, int storage, int smem_bytes) {
    switch (storage) {
        case 0: return prepare_st<0>(np, smem_bytes);
        case 1: return prepare_st<1>(np, smem_bytes);
        case 2: return prepare_st<2>(np, smem_bytes);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_forward_c64(const PlanImpl& p, const ChainArgs& a, cudaStream_t stream) {
    return launch_st<0>(p.n_fft, a, p.threads, stream);
}

cudaError_t launch_forward(const PlanImpl& p, const ChainArgs& a, cudaStream_t stream) {
    switch (p.storage) {
        case CBESSFM_C64: return launch_st<0>(p.n_fft, a, p.threads, stream);
        case CBESSFM_F16x4: return launch_st<1>(p.n_fft, a, p.threads, stream);
        case CBESSFM_BF16x4: return launch_st<2>(p.n_fft, a, p.threads, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cbessfm
