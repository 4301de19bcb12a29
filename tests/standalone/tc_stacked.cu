// Standalone check and timing of the tensor-core batch step with an operand read in place:
// 2^nnb x 2^nbeta batches of M x 32 outputs over K = 256 (split bf16 hi+lo), A read from
// 2^(nnb + nq) stored blocks, the block of batch (nonb, beta) selected by bits 0..nq-1 of
// the batch pattern closed[beta]; B per batch; complex64 output.  With nbeta = 12, nq = 10
// and M = 1024 it is the batch step of the 5x8-grid, 16-cycle sampling job; nbeta = 10,
// nq = 8 is the same step at a quarter of every array (about four batches per block both
// ways).  Prints the best of `reps` launches (stack list + tile kernel) and checks six
// outputs against FP64 sums of the split planes; exits 1 on a mismatch or error.
// usage: tc_stacked reps M_log2 variant(0 stacked 128, 1 stacked 64, 2 unstacked 64)
//                   layout(0 n lowest, 1 m lowest) nbeta nq nnb(default 2)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <random>
#include <cuda.h>
#include "../../paper_2112_15083_gb300/csrc/tc.cuh"

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("%s: %s\n", #x, cudaGetErrorString(e)); return 1; } } while (0)

__device__ __forceinline__ float val_of(unsigned long long i, unsigned salt) {
    unsigned h = (unsigned)(i * 2654435761ull) ^ (unsigned)(i >> 29) ^ salt;
    h *= 0x9E3779B1u;
    return (float)((h >> 9) & 1023) / 1024.0f - 0.5f;
}
// planes: [4][count] bf16, plane p = re_hi, re_lo, im_hi, im_lo of element i
__global__ void fill_split(__nv_bfloat16 *x, unsigned long long count, unsigned salt) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float re = val_of(2 * i, salt), im = val_of(2 * i + 1, salt);
        const __nv_bfloat16 rh = __float2bfloat16(re), ih = __float2bfloat16(im);
        x[i] = rh;
        x[count + i] = __float2bfloat16(re - __bfloat162float(rh));
        x[2 * count + i] = ih;
        x[3 * count + i] = __float2bfloat16(im - __bfloat162float(ih));
    }
}

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int encode(EncodeFn enc, CUtensorMap *m, void *base, int lk, int lrows, int lplanes_bat, int box_rows) {
    cuuint64_t dims[4] = {(cuuint64_t)1 << lk, (cuuint64_t)1 << lrows, (cuuint64_t)4 << lplanes_bat, 1};
    cuuint64_t strides[3] = {((cuuint64_t)1 << lk) * 2, ((cuuint64_t)1 << (lk + lrows)) * 2,
                             ((cuuint64_t)1 << (lk + lrows + lplanes_bat)) * 8};
    cuuint32_t box[4] = {(cuuint32_t)tnk::kTcBK, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { printf("encode failed %d\n", (int)r); return 1; }
    return 0;
}

int main(int argc, char **argv) {
    const int reps = argc > 1 ? atoi(argv[1]) : 10;
    const int lm = argc > 2 ? atoi(argv[2]) : 10;
    const int var = argc > 3 ? atoi(argv[3]) : 0;  // 0 stacked 128, 1 stacked 64, 2 plain 64
    const int nbeta = argc > 5 ? atoi(argv[5]) : 12, nq = argc > 6 ? atoi(argv[6]) : 10;
    const int nnb = argc > 7 ? atoi(argv[7]) : 2, ln = 5, lk = 8;
    if (reps < 1 || lm < 7 || lm > 12 || var < 0 || var > 2 || nbeta < 1 || nbeta > 14 || nq < 0 || nq > 20 || nnb < 0 || nnb > 4) {
        printf("usage: tc_stacked reps M_log2(7..12) variant(0..2) layout(0|1) nbeta(1..14) nq(0..20) nnb(0..4)\n");
        return 2;
    }
    const int lbat = nnb + nbeta, lba = nnb + nq, T = 1 << nbeta;
    const unsigned long long cA = 1ull << (lba + lm + lk), cB = 1ull << (lbat + ln + lk), cC = 1ull << (lbat + lm + ln);
    __nv_bfloat16 *A, *B;
    float2 *C;
    CK(cudaMalloc(&A, 4 * cA * 2));
    CK(cudaMalloc(&B, 4 * cB * 2));
    CK(cudaMalloc(&C, cC * 8));
    fill_split<<<4096, 256>>>(A, cA, 1u);
    fill_split<<<4096, 256>>>(B, cB, 2u);
    std::vector<unsigned long long> hclosed(T);
    std::mt19937_64 rng(7);
    for (auto &x : hclosed) x = rng();
    unsigned long long *dclosed;
    CK(cudaMalloc(&dclosed, T * 8));
    CK(cudaMemcpy(dclosed, hclosed.data(), T * 8, cudaMemcpyHostToDevice));
    int *vidx, *err, *stack;
    CK(cudaMalloc(&vidx, 8));
    CK(cudaMemset(vidx, 0, 8));
    CK(cudaMalloc(&err, 4));
    CK(cudaMemset(err, 0, 4));
    CK(cudaMalloc(&stack, (1 + 5 * T) * 4));
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q));
    EncodeFn enc = (EncodeFn)fn;
    CUtensorMap ma, mb32, mb64;
    if (encode(enc, &ma, A, lk, lm, lba, 128) || encode(enc, &mb32, B, lk, ln, lbat, 32) ||
        encode(enc, &mb64, B, lk, ln, lbat, 64))
        return 1;
    tnk::TcParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.C = C;
    tp.c_plane = (long long)cC;
    tp.vidx = vidx;
    tp.nver = 1;
    tp.lm = lm; tp.ln = ln; tp.lk = lk; tp.lbat = lbat;
    tp.out_fmt = tnk::OUT_C64;
    tp.out_scale = 1.f;
    tp.err = err;
    tp.group_m = 1;
    tp.ga.closed = reinterpret_cast<const uint64_t *>(dclosed);
    tp.ga.beta_mask = (1u << nbeta) - 1;
    for (int i = 0; i < nbeta; i++) tp.ga.beta_t[i] = (int8_t)i;
    tp.ga.nnb = nnb;
    tp.ga.nq = nq;
    for (int t = 0; t < nq; t++) tp.ga.q[t] = (int8_t)t;
    const int mlow = argc > 4 ? atoi(argv[4]) : 0;  // 1: C with m lowest, then n
    for (int i = 0; i < ln; i++) tp.pos_n[i] = (int8_t)(mlow ? lm + i : i);
    for (int i = 0; i < lm; i++) tp.pos_m[i] = (int8_t)(mlow ? i : ln + i);
    for (int i = 0; i < lbat; i++) tp.pos_bat[i] = (int8_t)(ln + lm + i);
    CK(cudaFuncSetAttribute(tnk::tc_cgemm<128, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tnk::TcSmem<128, 3>::kBytes));
    CK(cudaFuncSetAttribute(tnk::tc_cgemm<64, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, tnk::TcSmem<64, 4>::kBytes));
    CK(cudaFuncSetAttribute(tnk::tc_stack_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * T));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const long long tiles = (1LL << (lm - 7)) << lbat;
    const unsigned blocks = (unsigned)std::min<long long>(tiles, sms);
    auto launch = [&]() {
        if (var == 2) {
            tp.stack = nullptr;
            tnk::tc_cgemm<64, 4><<<blocks, tnk::kTcThreads, tnk::TcSmem<64, 4>::kBytes>>>(ma, mb64, tp);
            return;
        }
        const int BN = var == 0 ? 128 : 64;
        tp.stack = stack;
        tp.stack_S = BN >> ln;
        tnk::tc_stack_build<<<1, 1024, 8 * T>>>(tp.ga, nbeta, tp.stack_S, stack);
        if (var == 0) tnk::tc_cgemm<128, 3><<<blocks, tnk::kTcThreads, tnk::TcSmem<128, 3>::kBytes>>>(ma, mb32, tp);
        else tnk::tc_cgemm<64, 4><<<blocks, tnk::kTcThreads, tnk::TcSmem<64, 4>::kBytes>>>(ma, mb32, tp);
    };
    launch();
    CK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e9;
    for (int r = 0; r < reps; r++) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        best = ms < best ? ms : best;
    }
    int herr = 0, nst = 0;
    CK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&nst, stack, 4, cudaMemcpyDeviceToHost));
    const double bytes = (4.0 * cA * 2 + 4.0 * cB * 2 + cC * 8.0);
    printf("layout %s var %d lm %d: best %.3f ms, compulsory %.2f GB -> %.0f GB/s, stacks %d, err %d\n", mlow ? "m-low" : "n-low", var, lm, best, bytes / 1e9,
           bytes / best / 1e6, nst, herr);
    // spot checks against FP64 sums of the split planes
    const int K = 1 << lk;
    std::vector<__nv_bfloat16> pa(4 * K), pb(4 * K);
    double worst = 0;
    for (int s = 0; s < 6; s++) {
        const long long bat = (long long)(rng() % (1ull << lbat)), m = (long long)(rng() % (1ull << lm)),
                        n = (long long)(rng() % (1ull << ln));
        const long long beta = bat & (T - 1), nonb = bat >> nbeta;
        const long long z = nonb | ((long long)(hclosed[beta] & ((1ull << nq) - 1)) << nnb);
        for (int p = 0; p < 4; p++) {
            CK(cudaMemcpy(&pa[p * K], A + p * cA + (((z << lm) + m) << lk), K * 2, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(&pb[p * K], B + p * cB + (((bat << ln) + n) << lk), K * 2, cudaMemcpyDeviceToHost));
        }
        double re = 0, im = 0, mag = 0;
        for (int k = 0; k < K; k++) {
            const double ar = (double)__bfloat162float(pa[k]) + __bfloat162float(pa[K + k]);
            const double ai = (double)__bfloat162float(pa[2 * K + k]) + __bfloat162float(pa[3 * K + k]);
            const double br = (double)__bfloat162float(pb[k]) + __bfloat162float(pb[K + k]);
            const double bi = (double)__bfloat162float(pb[2 * K + k]) + __bfloat162float(pb[3 * K + k]);
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
            mag += (ar * ar + ai * ai) * (br * br + bi * bi);
        }
        float2 hc;
        CK(cudaMemcpy(&hc, C + (bat << (lm + ln)) + (mlow ? (n << lm) + m : (m << ln) + n), 8, cudaMemcpyDeviceToHost));
        const double d = std::hypot(hc.x - re, hc.y - im) / std::sqrt(mag);
        worst = d > worst ? d : worst;
    }
    const bool ok = worst < 1e-3 && herr == 0 && (var == 2 || nst > 0);
    printf("spot check: worst |c - ref| / sqrt(sum |a|^2 |b|^2) = %.2e %s\n", worst, ok ? "ok" : "MISMATCH");
    return ok ? 0 : 1;
}
