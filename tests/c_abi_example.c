/*
 * A plain C99 program that uses libcbessfm through include/cbessfm.h and the CUDA runtime only
 * (no Python): it reads a field and taps from files, backpropagates on the GPU, checks the
 * documented error paths, and writes the output.  tests/test_c_abi.py builds and runs it.
 *
 * usage: c_abi_example in.bin taps.bin out.bin bands steps ntaps n_fft overlap n_samples
 *                      ratio beta2 span_length n_spans sample_rate
 *   in.bin   n_samples 4D samples as float32 (x.re, x.im, y.re, y.im)
 *   taps.bin steps * bands * bands * ntaps float32 effective taps
 * exit status 0 on success, 1 on any failure (with a message on stderr).
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "cbessfm.h"

static int read_file(const char* path, void* dst, size_t bytes) {
    FILE* f = fopen(path, "rb");
    if (!f) return 0;
    const size_t got = fread(dst, 1, bytes, f);
    fclose(f);
    return got == bytes;
}

static int fail_msg(const char* what) {
    fprintf(stderr, "c_abi_example: %s (%s)\n", what, cbessfm_last_error());
    return 1;
}

int main(int argc, char** argv) {
    if (argc != 15) {
        fprintf(stderr, "c_abi_example: expected 14 arguments\n");
        return 1;
    }
    const int bands = atoi(argv[4]), steps = atoi(argv[5]), ntaps = atoi(argv[6]);
    const int n_fft = atoi(argv[7]), overlap = atoi(argv[8]);
    const long long n_samples = atoll(argv[9]);
    const double ratio = atof(argv[10]);
    cbessfm_link link;
    memset(&link, 0, sizeof(link));
    link.beta2 = atof(argv[11]);
    link.span_length = atof(argv[12]);
    link.n_spans = atoi(argv[13]);
    link.sample_rate = atof(argv[14]);

    const size_t field_bytes = (size_t)n_samples * 16;
    const size_t n_taps = (size_t)steps * bands * bands * ntaps;
    float* h_in = (float*)malloc(field_bytes);
    float* h_out = (float*)malloc(field_bytes);
    float* taps = (float*)malloc(n_taps * sizeof(float) + 4);
    if (!h_in || !h_out || !taps) return 1;
    if (!read_file(argv[1], h_in, field_bytes) || !read_file(argv[2], taps, n_taps * sizeof(float))) {
        fprintf(stderr, "c_abi_example: cannot read the input files\n");
        return 1;
    }

    cbessfm_plan* plan = NULL;
    if (cbessfm_plan_create(&link, bands, steps, ratio, taps, ntaps, n_fft, overlap, CBESSFM_C64,
                            &plan) != CBESSFM_OK)
        return fail_msg("plan_create");

    /* documented argument errors, before any device memory exists */
    if (cbessfm_backpropagate(plan, NULL, NULL, n_samples, 1, NULL) != CBESSFM_ERR_INVALID_ARG)
        return fail_msg("NULL buffers not rejected");
    if (strlen(cbessfm_last_error()) == 0) return fail_msg("no message for the rejected call");

    void* d_in = NULL;
    void* d_out = NULL;
    if (cudaMalloc(&d_in, field_bytes) != cudaSuccess || cudaMalloc(&d_out, field_bytes) != cudaSuccess)
        return fail_msg("cudaMalloc");
    if (cudaMemcpy(d_in, h_in, field_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail_msg("copy in");
    if (cbessfm_backpropagate(plan, d_in, d_in, n_samples, 1, NULL) != CBESSFM_ERR_ALIAS)
        return fail_msg("aliased output not rejected");
    if (cbessfm_backpropagate(plan, d_in, d_out, n_samples, 1, NULL) != CBESSFM_OK)
        return fail_msg("backpropagate");
    if (cudaDeviceSynchronize() != cudaSuccess) return fail_msg("synchronize");
    if (cbessfm_get_status(plan, NULL) != CBESSFM_OK) return fail_msg("device status");
    if (cudaMemcpy(h_out, d_out, field_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail_msg("copy out");

    FILE* f = fopen(argv[3], "wb");
    if (!f || fwrite(h_out, 1, field_bytes, f) != field_bytes) return fail_msg("write output");
    fclose(f);
    cudaFree(d_in);
    cudaFree(d_out);
    if (cbessfm_plan_destroy(plan) != CBESSFM_OK) return fail_msg("plan_destroy");
    free(h_in);
    free(h_out);
    free(taps);
    printf("c_abi_example: ok (%s)\n", cbessfm_version());
    return 0;
}
