// Standalone check and timing of the long-K kernel on 2^lbat batches of 64 x 8 outputs over
// K = 2048 (complex64; with lbat = 12 the root product of the 5x8-grid, 16-cycle sampling
// job), synthetic data, no gathers.  Prints the best of `reps` launches and checks one output
// against an FP64 host sum; exits 1 on a mismatch or error.
// usage: long_k reps lbat variant(0: 8 warps x 4 rows, 1: 16 x 2 (the engine's), 2: 32 x 1)
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include "../../paper_2112_15083_gb300/csrc/kernels.cuh"

__global__ void fill(float2 *x, size_t n, float s) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = make_float2(__sinf(s * (float)(i & 65535)), __cosf(s * (float)(i & 4095)));
}

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("%s: %s\n", #x, cudaGetErrorString(e)); return 1; } } while (0)

int main(int argc, char **argv) {
    const int lbat = argc > 2 ? atoi(argv[2]) : 12, lm = 6, ln = 3, lk = 11;
    if (lbat < 3 || lbat > 14) {
        printf("usage: long_k reps lbat(3..14) variant(0..2)\n");
        return 2;
    }
    const size_t nA = 1ull << (lbat + lm + lk), nB = 1ull << (lbat + ln + lk), nC = 1ull << (lbat + lm + ln);
    float2 *A, *B, *C;
    CK(cudaMalloc(&A, nA * 8));
    CK(cudaMalloc(&B, nB * 8));
    CK(cudaMalloc(&C, nC * 8));
    fill<<<1024, 256>>>(A, nA, 0.001f);
    fill<<<1024, 256>>>(B, nB, 0.002f);
    const void **dpa, **dpb;
    CK(cudaMalloc(&dpa, 8));
    CK(cudaMalloc(&dpb, 8));
    CK(cudaMemcpy(dpa, &A, 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dpb, &B, 8, cudaMemcpyHostToDevice));
    int *err;
    CK(cudaMalloc(&err, 4));
    CK(cudaMemset(err, 0, 4));
    tnk::GemmParams p;
    memset(&p, 0, sizeof(p));
    p.ptrA = reinterpret_cast<const void *const *>(dpa);
    p.ptrB = reinterpret_cast<const void *const *>(dpb);
    p.C = C;
    p.c_vstride = (long long)nC;
    p.nver = 1;
    p.lm = lm; p.ln = ln; p.lk = lk; p.lbat = lbat;
    p.out_fmt = tnk::OUT_C64;
    p.out_scale = 1.f;
    p.err = err;
    for (int i = 0; i < ln; i++) p.pos_n[i] = i;
    for (int i = 0; i < lm; i++) p.pos_m[i] = ln + i;
    for (int i = 0; i < lbat; i++) p.pos_bat[i] = ln + lm + i;
    const int var = argc > 3 ? atoi(argv[3]) : 1;
    auto kern = var == 2 ? tnk::cgemm_skinny<32, 1, 8> : var == 1 ? tnk::cgemm_skinny<16, 2, 8> : tnk::cgemm_skinny<8, 4, 8>;
    const int threads = var == 2 ? 1024 : var == 1 ? 512 : 256;
    const int smem = tnk::kSkinnyST * tnk::skinny_stage_bytes<8, 4, 8>();  // same rows per block
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0, sms = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const long long units = (1LL << lbat) * 2;
    const int reps = argc > 1 ? atoi(argv[1]) : 10;
    const unsigned blocks = (unsigned)std::min<long long>(units, (long long)per_sm * sms);
    printf("var %d threads %d per_sm %d blocks %u smem %d\n", var, threads, per_sm, blocks, smem);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kern<<<blocks, threads, smem>>>(p);
    CK(cudaDeviceSynchronize());
    float best = 1e9;
    for (int r = 0; r < reps; r++) {
        cudaEventRecord(e0);
        kern<<<blocks, threads, smem>>>(p);
        cudaEventRecord(e1);
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        best = ms < best ? ms : best;
    }
    int herr = 0;
    CK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
    // spot check: output (bat 5, m 3, n 2) against a host sum
    float2 hc;
    const long long bat = 5, m = 3, n = 2;
    CK(cudaMemcpy(&hc, C + ((bat << (lm + ln)) | (m << ln) | n), 8, cudaMemcpyDeviceToHost));
    const int K = 1 << lk;
    float2 *ha = (float2 *)malloc(K * 8), *hb = (float2 *)malloc(K * 8);
    CK(cudaMemcpy(ha, A + (((bat << lm) | m) << lk), K * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hb, B + (((bat << ln) | n) << lk), K * 8, cudaMemcpyDeviceToHost));
    double re = 0, im = 0;
    for (int k = 0; k < K; k++) {
        re += (double)ha[k].x * hb[k].x - (double)ha[k].y * hb[k].y;
        im += (double)ha[k].x * hb[k].y + (double)ha[k].y * hb[k].x;
    }
    const double gb = (nA + nB) * 8.0 / 1e9;
    double mag = 0;
    for (int k = 0; k < K; k++)
        mag += ((double)ha[k].x * ha[k].x + (double)ha[k].y * ha[k].y) * ((double)hb[k].x * hb[k].x + (double)hb[k].y * hb[k].y);
    const double rel = std::hypot(hc.x - re, hc.y - im) / std::sqrt(mag);
    const bool ok = herr == 0 && rel < 1e-5;
    printf("best %.3f ms  %.0f GB/s  err %d  check (%.4f, %.4f) vs (%.4f, %.4f) rel %.1e %s\n", best, gb / best * 1e3, herr,
           hc.x, hc.y, re, im, rel, ok ? "ok" : "MISMATCH");
    return ok ? 0 : 1;
}
