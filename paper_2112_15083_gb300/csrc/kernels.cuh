// Device kernels of libtn (sm_103a).
//
//  * cgemm_row / cgemm_tile: one pairwise contraction step (Sec. I, contraction tree;
//    the per-slice work of Sec. I.C) as a batched complex GEMM
//        C[v][bat][m][n] = sum_k A[v][bat][m][k] * B[v][bat][n][k]
//    over versions v (slice assignments of the sliced legs the operands depend on),
//    with the permutation of the result fused into the epilogue: element (bat, m, n)
//    goes to bit-scattered address pos_bat(bat) + pos_m(m) + pos_n(n).
//  * materialize: writes leaf tensors in the layout their consumer reads, fixing the
//    sliced legs (one copy per slice value) and binding closed output legs to the
//    batch pattern (the batch-indexed selector <b_B|).
//  * slice_sum: FP64 sum over the slice set in slice order (Sec. I.C step 1);
//    root_slice_sum: the same sum fused with a root step that runs the row kernel.
//  * draw / sampler: Philox4x32-10 draws and the modified frugal rejection step
//    (Sec. II.A), one warp per batch of 64.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "widen.h"

namespace tnk {

constexpr int kMaxBits = 40;

// Storage formats of a tensor (chosen by the kernel that reads it): interleaved
// complex64, or four planes (re_hi, re_lo, im_hi, im_lo) of bf16 / fp16 with x = hi + lo,
// plane stride = the tensor's element count.  Both use 8 bytes per element.
enum OutFmt { OUT_C64 = 0, OUT_SPLIT_BF16 = 1, OUT_SPLIT_FP16 = 2 };

// A step operand whose closed output legs are selected per batch.  src stores the
// operand with its nq closed legs as the top bits (every value of those legs, shared by
// all batches); dst is the operand as the step reads it: nbits layout bits of which the
// beta bits sit at pos_beta[t] and the other nbits - lb bits are src's low bits in order.
// dst element e of batch beta = src element (sel << (nbits - lb)) | rest(e), where sel
// packs the batch pattern's bits q[0], q[1], ... (closed positions).
struct GatherDesc {
    const char *src;
    char *dst;
    long long nver;              // versions (each: nplanes planes)
    long long src_plane, dst_plane;  // elements per plane
    int nplanes, esize;          // 4 x 2 B (split) or 1 x 8 B / 16 B
    int nbits, lb, nq;
    int vec_log2;                // log2 of elements per 16-byte chunk (0 when runs are shorter)
    int run_log2;                // log2 of chunks per run: dst positions below the lowest beta
                                 // position, where batch and selection stay constant
    int8_t pos_beta[16];         // beta bit t -> dst position, sorted by descending position
    int8_t beta_bit[16];         // ... and which beta bit sits there
    int16_t q[32];
    // byte lookup tables of the same maps (built on the host): for byte j of e and value x,
    // rest_tab[j][x] and beta_tab[j][x] are the contributions of x << 8j to the source's low
    // bits and to the batch index; sel_tab[j][x] that of byte j of the batch pattern
    const uint64_t *rest_tab;    // [5][256]
    const uint32_t *beta_tab;    // [5][256]
    const uint32_t *sel_tab;     // [8][256]
};
constexpr int kGatherTabWords = 5 * 256 + (5 * 256 + 8 * 256) / 2;  // 64-bit words per gather

// Source element of dst element e (a run's first element in the run path).
__device__ __forceinline__ long long gather_src(const GatherDesc &d, long long e, const uint64_t *closed_bits) {
    uint64_t rest = 0;
    uint32_t beta = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const uint32_t x = (uint32_t)(e >> (8 * j)) & 255u;
        rest |= __ldg(&d.rest_tab[j * 256 + x]);
        beta |= __ldg(&d.beta_tab[j * 256 + x]);
    }
    const uint64_t pat = closed_bits[beta];
    uint64_t sel = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) sel |= __ldg(&d.sel_tab[j * 256 + (uint32_t)((pat >> (8 * j)) & 255u)]);
    return (long long)((sel << (d.nbits - d.lb)) | rest);
}

struct GemmParams {
    const void *const *ptrA;  // per C-version operand base
    const void *const *ptrB;
    void *C;                  // C base (version v at C + v * c_vstride elements)
    long long c_vstride;      // elements
    long long nver;
    int lm, ln, lk, lbat;     // log2 of M, N, K, BAT
    int out_fmt;              // OutFmt of C
    float out_scale;          // multiplier applied before storing
    int swapped;              // operands exchanged (A holds the step's B): keep the step's
                              // operand order inside each complex multiply-add
    // row kernel only: operands read through their batch gather instead of a gathered
    // copy (null: not gathered); closed_bits are the group's batch patterns
    const GatherDesc *gA, *gB;
    const uint64_t *closed_bits;
    int *err;                 // long-K kernel: set to 1 if a bounded wait gives up
    int8_t pos_bat[kMaxBits], pos_m[kMaxBits], pos_n[kMaxBits];
};

// Split x into hi + lo in the operand type and store both parts at plane stride.
__device__ __forceinline__ void store_split(void *base, long long plane, long long off, float2 x, bool fp16) {
    if (fp16) {
        __half *h = static_cast<__half *>(base);
        const __half rh = __float2half_rn(x.x), ih = __float2half_rn(x.y);
        h[off] = rh;
        h[plane + off] = __float2half_rn(x.x - __half2float(rh));
        h[2 * plane + off] = ih;
        h[3 * plane + off] = __float2half_rn(x.y - __half2float(ih));
    } else {
        __nv_bfloat16 *h = static_cast<__nv_bfloat16 *>(base);
        const __nv_bfloat16 rh = __float2bfloat16_rn(x.x), ih = __float2bfloat16_rn(x.y);
        h[off] = rh;
        h[plane + off] = __float2bfloat16_rn(x.x - __bfloat162float(rh));
        h[2 * plane + off] = ih;
        h[3 * plane + off] = __float2bfloat16_rn(x.y - __bfloat162float(ih));
    }
}

// Store one complex64 result of version v in C's format.
__device__ __forceinline__ void store_c(const GemmParams &p, long long v, long long off, float2 x) {
    x.x *= p.out_scale;
    x.y *= p.out_scale;
    if (p.out_fmt == OUT_C64) {
        static_cast<float2 *>(p.C)[v * p.c_vstride + off] = x;
    } else {
        unsigned short *base = static_cast<unsigned short *>(p.C) + 4 * v * p.c_vstride;
        store_split(base, p.c_vstride, off, x, p.out_fmt == OUT_SPLIT_FP16);
    }
}
template <typename T> __device__ __forceinline__ void store_c_t(const GemmParams &p, long long v, long long off, T x);
template <> __device__ __forceinline__ void store_c_t<float2>(const GemmParams &p, long long v, long long off, float2 x) {
    store_c(p, v, off, x);
}
template <> __device__ __forceinline__ void store_c_t<double2>(const GemmParams &p, long long v, long long off, double2 x) {
    static_cast<double2 *>(p.C)[v * p.c_vstride + off] = x;
}

__device__ __forceinline__ long long scatter_bits(long long x, const int8_t *pos, int nbits) {
    long long off = 0;
#pragma unroll 4
    for (int i = 0; i < nbits; i++) off |= ((x >> i) & 1LL) << pos[i];
    return off;
}

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}
template <typename T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

// One output row (v, bat, m) per thread and call; all N (<= 32) columns in registers.  For the
// gate-absorption steps (small N and K), which are bound by HBM bandwidth.
// Offset of a gathered operand's element e in its shared storage.  Lanes of a warp whose
// elements share the batch and selection (same e >> shift) take the leader's decode.
__device__ __forceinline__ long long gather_src_warp(const GatherDesc &d, long long e, int shift,
                                                     const uint64_t *closed_bits) {
    const unsigned mask = __activemask();
    const int leader = __ffs(mask) - 1;
    const long long e0 = __shfl_sync(mask, e, leader);
    if (__all_sync(mask, (e >> shift) == (e0 >> shift))) {
        long long s0 = 0;
        if ((int)(threadIdx.x & 31) == leader) s0 = gather_src(d, e0, closed_bits);
        s0 = __shfl_sync(mask, s0, leader);
        return s0 + (e - e0);
    }
    return gather_src(d, e, closed_bits);
}

template <typename T, int N>
__device__ __forceinline__ void cgemm_row_one(const GemmParams &p, long long row) {
    const long long M = 1LL << p.lm;
    const long long m = row & (M - 1);
    const long long bat = (row >> p.lm) & ((1LL << p.lbat) - 1);
    const long long v = row >> (p.lm + p.lbat);
    const int K = 1 << p.lk;
    const T *A, *B;
    if (p.gA) {
        const long long e = ((bat << p.lm) | m) << p.lk;
        A = reinterpret_cast<const T *>(p.gA->src) + gather_src_warp(*p.gA, e, p.gA->pos_beta[p.gA->lb - 1], p.closed_bits);
    } else {
        A = static_cast<const T *>(p.ptrA[v]) + (((bat << p.lm) | m) << p.lk);
    }
    if (p.gB) {
        const long long e = bat << (p.ln + p.lk);
        B = reinterpret_cast<const T *>(p.gB->src) + gather_src_warp(*p.gB, e, p.gB->pos_beta[p.gB->lb - 1], p.closed_bits);
    } else {
        B = static_cast<const T *>(p.ptrB[v]) + (bat << (p.ln + p.lk));
    }
    T acc[N];
#pragma unroll
    for (int n = 0; n < N; n++) acc[n] = czero<T>();
    // complex64 rows of even K are read 16 bytes (two elements) at a time; the
    // accumulation order over k is the same either way
    auto step = [&](const T a, int k) {
        if (p.swapped) {
#pragma unroll
            for (int n = 0; n < N; n++) acc[n] = cfma(__ldg(&B[(n << p.lk) + k]), a, acc[n]);
        } else {
#pragma unroll
            for (int n = 0; n < N; n++) acc[n] = cfma(a, __ldg(&B[(n << p.lk) + k]), acc[n]);
        }
    };
    if constexpr (sizeof(T) == 8) {
        if (K >= 2) {
            for (int k = 0; k < K; k += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(A + k);
                step(make_float2(v.x, v.y), k);
                step(make_float2(v.z, v.w), k + 1);
            }
        } else {
            step(A[0], 0);
        }
    } else {
        for (int k = 0; k < K; k++) step(A[k], k);
    }
    const long long cb = scatter_bits(bat, p.pos_bat, p.lbat) + scatter_bits(m, p.pos_m, p.lm);
#pragma unroll
    for (int n = 0; n < N; n++) store_c_t<T>(p, v, cb + scatter_bits(n, p.pos_n, p.ln), acc[n]);
}

// Grid-stride over rows (the grid is bounded by the launch).
template <typename T, int N>
__global__ void __launch_bounds__(256) cgemm_row(GemmParams p) {
    const long long rows = p.nver << (p.lbat + p.lm);
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (long long)gridDim.x * blockDim.x)
        cgemm_row_one<T, N>(p, row);
}

// The row kernel with coalesced row reads, for complex64 rows of 16 <= K <= 64: each warp
// copies its 32 rows into shared memory (K/2 lanes per row, 16 bytes each, 64/K rows per
// load instruction), then each lane forms its own row's N outputs exactly as cgemm_row_one
// does (the same k order and multiply-add operand order), so the results are
// bit-identical.  Rows sit kRowPad bytes apart beyond their length, which keeps the lanes'
// 16-byte shared reads free of bank conflicts.
constexpr int kRowWarps = 4;     // warps per block
constexpr int kRowPad = 16;      // bytes between staged rows
template <int N>
__global__ void __launch_bounds__(32 * kRowWarps) cgemm_rowstage(GemmParams p) {
    extern __shared__ __align__(16) unsigned char rowstage_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = 1 << p.lk;
    const int rstride = 8 * K + kRowPad;  // bytes
    unsigned char *stage = rowstage_smem + (size_t)warp * 32 * rstride;
    const long long M = 1LL << p.lm;
    const long long rows = p.nver << (p.lbat + p.lm);
    const int lpr = K >> 1;         // lanes per row (16 bytes = two complex64 each)
    const int rpi = 32 / lpr;       // rows per load instruction
    for (long long r0 = ((long long)blockIdx.x * kRowWarps + warp) * 32; r0 < rows;
         r0 += (long long)gridDim.x * kRowWarps * 32) {
        // this lane's row and its operand bases
        const long long row = r0 + lane;
        const bool live = row < rows;
        const long long m = row & (M - 1);
        const long long bat = (row >> p.lm) & ((1LL << p.lbat) - 1);
        const long long v = row >> (p.lm + p.lbat);
        const float2 *A = nullptr, *B = nullptr;
        if (live) {
            if (p.gA) {
                const long long e = ((bat << p.lm) | m) << p.lk;
                A = reinterpret_cast<const float2 *>(p.gA->src) +
                    gather_src_warp(*p.gA, e, p.gA->pos_beta[p.gA->lb - 1], p.closed_bits);
            } else {
                A = static_cast<const float2 *>(p.ptrA[v]) + (((bat << p.lm) | m) << p.lk);
            }
            if (p.gB) {
                const long long e = bat << (p.ln + p.lk);
                B = reinterpret_cast<const float2 *>(p.gB->src) +
                    gather_src_warp(*p.gB, e, p.gB->pos_beta[p.gB->lb - 1], p.closed_bits);
            } else {
                B = static_cast<const float2 *>(p.ptrB[v]) + (bat << (p.ln + p.lk));
            }
        }
        // stage the warp's rows: in instruction j, lane l copies chunk l % lpr of row
        // j * rpi + l / lpr
        const unsigned long long abase = reinterpret_cast<unsigned long long>(A);
        for (int j = 0; j < 32; j += rpi) {
            const int rr = j + lane / lpr;
            const unsigned long long src = __shfl_sync(0xffffffffu, abase, rr);
            if (r0 + rr < rows) {
                const int c = lane % lpr;
                const float4 x = *reinterpret_cast<const float4 *>(src + 16ull * c);
                *reinterpret_cast<float4 *>(stage + (size_t)rr * rstride + 16 * c) = x;
            }
        }
        __syncwarp();
        if (live) {
            const float2 *a = reinterpret_cast<const float2 *>(stage + (size_t)lane * rstride);
            float2 acc[N];
#pragma unroll
            for (int n = 0; n < N; n++) acc[n] = czero<float2>();
            for (int k = 0; k < K; k += 2) {
                const float4 q = *reinterpret_cast<const float4 *>(a + k);
                const float2 x0 = make_float2(q.x, q.y), x1 = make_float2(q.z, q.w);
                if (p.swapped) {
#pragma unroll
                    for (int n = 0; n < N; n++) acc[n] = cfma(__ldg(&B[(n << p.lk) + k]), x0, acc[n]);
#pragma unroll
                    for (int n = 0; n < N; n++) acc[n] = cfma(__ldg(&B[(n << p.lk) + k + 1]), x1, acc[n]);
                } else {
#pragma unroll
                    for (int n = 0; n < N; n++) acc[n] = cfma(x0, __ldg(&B[(n << p.lk) + k]), acc[n]);
#pragma unroll
                    for (int n = 0; n < N; n++) acc[n] = cfma(x1, __ldg(&B[(n << p.lk) + k + 1]), acc[n]);
                }
            }
            const long long cb = scatter_bits(bat, p.pos_bat, p.lbat) + scatter_bits(m, p.pos_m, p.lm);
#pragma unroll
            for (int n = 0; n < N; n++) store_c_t<float2>(p, v, cb + scatter_bits(n, p.pos_n, p.ln), acc[n]);
        }
        __syncwarp();  // the stage is rewritten by the next iteration
    }
}

// mbarrier primitives (shared-memory barriers with transaction counts).
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~limit cycles or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          long long limit) {
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}

// Bounded wait that ignores the abort flag (used to drain work already issued).
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) global -> shared,
// completing on mbarrier `bar` as transaction bytes.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Batched products with at most 64 rows and 8 columns and a long K (K >= 1024, complex64
// operands).  A block of W warps takes R = W MW rows of one (version, batch) at a time (a
// batch with more rows is split into row blocks); each warp owns MW rows of A and every
// column.  The block's work is one sequence of stages, each a (unit, K block of 64 U
// elements) pair, streamed through a ring of ST shared-memory stages by the bulk-copy
// engine (one contiguous copy per row and stage, issued ST - 1 stages ahead across unit
// boundaries and completing on the stage's mbarrier), so loads stay in flight while the
// FMAs run.  In a stage lane l reads elements 2 l and 2 l + 1 of each 64-element block of
// its warp's A rows; the stage's B rows are shared by the block.  Every wait is bounded:
// on timeout the block sets *err, lets its copies in flight land (bounded) and returns.
// Each lane accumulates in ascending k and the warp adds its 32 lane sums by a fixed xor
// butterfly.  Gathered operands are read in place, one decode per row and warp.  The lane
// split of K rounds differently from the kernels that accumulate each output over k in
// one thread, so it is the only kernel the engine runs for these shapes.
constexpr int kSkinnyU = 2;   // 64-element K blocks per stage
constexpr int kSkinnyST = 4;  // ring stages
template <int W, int MW, int N>
constexpr int skinny_stage_bytes() {
    return (W * MW + N) * kSkinnyU * 32 * 16;
}
template <int W, int MW, int N>
__global__ void __launch_bounds__(32 * W) cgemm_skinny(GemmParams p) {
    extern __shared__ float4 skinny_ring[];
    __shared__ __align__(8) uint64_t full[kSkinnyST];  // per stage: W arrivals + the bytes
    __shared__ int abort_flag;
    constexpr int R = W * MW, U = kSkinnyU, ST = kSkinnyST, NB = (N + W - 1) / W;
    const long long kLimit = 4000000000LL;
    constexpr int kStage = (R + N) * U * 32;  // float4 per stage
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row_blocks = (1 << p.lm) / R;
    const long long units = (p.nver << p.lbat) * row_blocks;
    const int nk = (1 << p.lk) / (64 * U);  // stages per unit
    const long long mine = units > blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long total = mine * nk;
    // copy side: the row pointers of the unit being issued
    const float2 *a[MW], *b[NB];
    long long a_unit = -1;
    auto unit_of = [&](long long ul, long long &bat, long long &v, int &row0) {
        const long long u = blockIdx.x + ul * gridDim.x;
        const int rb = (int)(u % row_blocks);
        const long long bv = u / row_blocks;
        bat = bv & ((1LL << p.lbat) - 1);
        v = bv >> p.lbat;
        row0 = rb * R + warp * MW;  // this warp's first row of A
    };
    // copies of stage (unit ul, K block kb) into ring slot `slot`
    auto issue = [&](long long ul, int kb, int slot) {
        if (ul != a_unit) {
            long long bat, v;
            int row0;
            unit_of(ul, bat, v, row0);
#pragma unroll
            for (int i = 0; i < MW; i++) {
                const long long e = ((bat << p.lm) | (long long)(row0 + i)) << p.lk;
                a[i] = p.gA ? reinterpret_cast<const float2 *>(p.gA->src) +
                                  gather_src_warp(*p.gA, e, p.gA->pos_beta[p.gA->lb - 1], p.closed_bits)
                            : static_cast<const float2 *>(p.ptrA[v]) + e;
            }
#pragma unroll
            for (int r = 0; r < NB; r++) {
                const int n = warp + r * W;
                const long long e = (bat << (p.ln + p.lk)) | ((long long)(n < N ? n : 0) << p.lk);
                b[r] = p.gB ? reinterpret_cast<const float2 *>(p.gB->src) +
                                  gather_src_warp(*p.gB, e, p.gB->pos_beta[p.gB->lb - 1], p.closed_bits)
                            : static_cast<const float2 *>(p.ptrB[v]) + e;
            }
            a_unit = ul;
        }
        // lane 0 of each warp: one arrival with the warp's bytes, then its rows' copies
        if (lane == 0) {
            float4 *st = skinny_ring + slot * kStage;
            const uint32_t bar = smem_u32(&full[slot]);
            int rows = MW;
#pragma unroll
            for (int r = 0; r < NB; r++) rows += warp + r * W < N;
            mbar_expect_tx(bar, (uint32_t)(rows * U * 512));
            const int k0 = kb * 64 * U;
#pragma unroll
            for (int i = 0; i < MW; i++) bulk_load(&st[(warp * MW + i) * U * 32], a[i] + k0, U * 512, bar);
#pragma unroll
            for (int r = 0; r < NB; r++)
                if (warp + r * W < N) bulk_load(&st[(R + warp + r * W) * U * 32], b[r] + k0, U * 512, bar);
        }
    };
    float2 acc[MW][N];
#pragma unroll
    for (int i = 0; i < MW; i++)
#pragma unroll
        for (int n = 0; n < N; n++) acc[i][n] = make_float2(0.f, 0.f);
    if (threadIdx.x == 0) {
        for (int i = 0; i < ST; i++) mbar_init(smem_u32(&full[i]), W);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // stage counters advance by one (no divisions in the loop): issue side (iul, ikb, islot)
    // runs ST - 1 stages ahead of the compute side (ul, kb, slot, parity)
    long long issued = 0, iul = 0;
    int ikb = 0, islot = 0;
    auto advance_issue = [&]() {
        issued++;
        if (++ikb == nk) { ikb = 0; iul++; }
        if (++islot == ST) islot = 0;
    };
    for (; issued < ST - 1 && issued < total;) {
        issue(iul, ikb, islot);
        advance_issue();
    }
    long long g = 0, ul = 0;
    int kb = 0, slot = 0;
    uint32_t parity = 0;
    for (; g < total; g++) {
        __syncthreads();  // every warp is done with the slot the next issue overwrites
        if (issued < total) {
            issue(iul, ikb, islot);
            advance_issue();
        }
        mbar_wait(smem_u32(&full[slot]), parity, &abort_flag, kLimit);
        __syncthreads();  // a timeout anywhere ends the block's loop in every thread
        if (abort_flag) break;
        const float4 *st = skinny_ring + slot * kStage;
        if (++slot == ST) { slot = 0; parity ^= 1u; }
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int n = 0; n < N; n++) {
                const float4 yb = st[((R + n) * U + u) * 32 + lane];
#pragma unroll
                for (int i = 0; i < MW; i++) {
                    const float4 x = st[((warp * MW + i) * U + u) * 32 + lane];
                    acc[i][n] = cfma(make_float2(x.x, x.y), make_float2(yb.x, yb.y), acc[i][n]);
                    acc[i][n] = cfma(make_float2(x.z, x.w), make_float2(yb.z, yb.w), acc[i][n]);
                }
            }
        if (++kb < nk) continue;
        kb = 0;
        // the unit's last stage: reduce, store, start the next unit from zero
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int i = 0; i < MW; i++)
#pragma unroll
                for (int n = 0; n < N; n++) {
                    acc[i][n].x += __shfl_xor_sync(0xffffffffu, acc[i][n].x, off);
                    acc[i][n].y += __shfl_xor_sync(0xffffffffu, acc[i][n].y, off);
                }
        long long bat, v;
        int row0;
        unit_of(ul++, bat, v, row0);
        // every lane holds the totals: lane i N + n stores output (row MW warp + i, column n)
        const long long cb = scatter_bits(bat, p.pos_bat, p.lbat);
#pragma unroll
        for (int i = 0; i < MW; i++)
#pragma unroll
            for (int n = 0; n < N; n++) {
                if (lane == i * N + n)
                    store_c(p, v, cb + scatter_bits(row0 + i, p.pos_m, p.lm) + scatter_bits(n, p.pos_n, p.ln),
                            acc[i][n]);
                acc[i][n] = make_float2(0.f, 0.f);
            }
    }
    if (abort_flag && threadIdx.x == 0) {
        atomicExch(p.err, 1);
        // let the copies already issued land before the shared memory is released
        for (long long q = g; q < issued; q++) mbar_drain(smem_u32(&full[q % ST]), (uint32_t)((q / ST) & 1), kLimit);
    }
    __syncthreads();
}

// Batched small products (M, N <= 64, K <= 64): a block stages the operands of 2^lg
// consecutive batches in shared memory and walks that chunk's outputs in the order of
// their positions in C (local bit i = chunk bit kind[i] / idx[i]), so consecutive threads
// store to consecutive addresses whenever C's lowest positions lie in the chunk.
struct SmallMap {
    int lg;              // log2 batches per block
    int nloc;            // lg + lm + ln
    int8_t kind[48];     // 0: batch bit, 1: m bit, 2: n bit
    int8_t idx[48];
};

template <typename T>
__global__ void __launch_bounds__(256) cgemm_small(GemmParams p, SmallMap smp) {
    extern __shared__ __align__(16) unsigned char small_smem[];
    __shared__ SmallMap sm;  // its tables are read per output
    if (threadIdx.x == 0) sm = smp;
    T *As = reinterpret_cast<T *>(small_smem);
    const int M = 1 << p.lm, N = 1 << p.ln, K = 1 << p.lk, G = 1 << smp.lg;
    const int KP = K + 1;  // padded row: rows of consecutive outputs fall in different banks
    T *Bs = As + (size_t)G * M * KP;
    const long long chunks = 1LL << (p.lbat - smp.lg);
    const long long v = (long long)blockIdx.x / chunks;
    const long long bat0 = ((long long)blockIdx.x - v * chunks) << smp.lg;
    if (v >= p.nver) return;
    const T *A = static_cast<const T *>(p.ptrA[v]) + (bat0 << (p.lm + p.lk));
    const T *B = static_cast<const T *>(p.ptrB[v]) + (bat0 << (p.ln + p.lk));
    for (int e = threadIdx.x; e < G * M * K; e += blockDim.x) As[(e >> p.lk) * KP + (e & (K - 1))] = A[e];
    for (int e = threadIdx.x; e < G * N * K; e += blockDim.x) Bs[(e >> p.lk) * KP + (e & (K - 1))] = B[e];
    __syncthreads();
    const long long cbase = scatter_bits(bat0, p.pos_bat, p.lbat);
    const int nout = G * M * N;
    for (int l = threadIdx.x; l < nout; l += blockDim.x) {
        int b = 0, m = 0, n = 0;
        for (int i = 0; i < sm.nloc; i++) {
            const int bit = (l >> i) & 1;
            if (sm.kind[i] == 0) b |= bit << sm.idx[i];
            else if (sm.kind[i] == 1) m |= bit << sm.idx[i];
            else n |= bit << sm.idx[i];
        }
        const T *a = As + (size_t)(b * M + m) * KP;
        const T *bb = Bs + (size_t)(b * N + n) * KP;
        T acc = czero<T>();
        for (int k = 0; k < K; k++) acc = cfma(a[k], bb[k], acc);
        const long long off = cbase + scatter_bits(b, p.pos_bat, smp.lg) + scatter_bits(m, p.pos_m, p.lm) +
                              scatter_bits(n, p.pos_n, p.ln);
        store_c_t<T>(p, v, off, acc);
    }
}

// Shared-memory tiled kernel: TM x TN output tile, K in chunks of TK, each thread an
// RM x RN register tile (rows contiguous, columns strided by TN/RN for coalescing).
template <typename T, int TM, int TN, int TK, int RM, int RN>
__global__ void __launch_bounds__((TM / RM) * (TN / RN)) cgemm_tile(GemmParams p) {
    constexpr int NTX = TN / RN, NTY = TM / RM, NT = NTX * NTY;
    __shared__ T As[TK][TM + 1];
    __shared__ T Bs[TK][TN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % NTX, ty = tid / NTX;
    const long long M = 1LL << p.lm, N = 1LL << p.ln;
    const int K = 1 << p.lk;
    const int ltm = p.lm > 0 ? min(p.lm, __ffs(TM) - 1) : 0;
    const int ltn = p.ln > 0 ? min(p.ln, __ffs(TN) - 1) : 0;
    const int ltiles_m = p.lm - ltm, ltiles_n = p.ln - ltn;
    long long bid = blockIdx.x;
    const long long tn_i = bid & ((1LL << ltiles_n) - 1);
    bid >>= ltiles_n;
    const long long tm_i = bid & ((1LL << ltiles_m) - 1);
    bid >>= ltiles_m;
    const long long bat = bid & ((1LL << p.lbat) - 1);
    const long long v = bid >> p.lbat;
    if (v >= p.nver) return;
    const long long m0 = tm_i * TM, n0 = tn_i * TN;
    const int mrows = (int)min((long long)TM, M - m0), ncols = (int)min((long long)TN, N - n0);
    const T *A = static_cast<const T *>(p.ptrA[v]) + (((bat << p.lm) | m0) << p.lk);
    const T *B = static_cast<const T *>(p.ptrB[v]) + (((bat << p.ln) | n0) << p.lk);
    T acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; i++)
#pragma unroll
        for (int j = 0; j < RN; j++) acc[i][j] = czero<T>();
    const int kt = min(TK, K);
    const int lkt = __ffs(kt) - 1;
    for (int k0 = 0; k0 < K; k0 += kt) {
        for (int e = tid; e < (TM << lkt); e += NT) {
            int r = e >> lkt, c = e & (kt - 1);
            As[c][r] = r < mrows ? A[((long long)r << p.lk) + k0 + c] : czero<T>();
        }
        for (int e = tid; e < (TN << lkt); e += NT) {
            int r = e >> lkt, c = e & (kt - 1);
            Bs[c][r] = r < ncols ? B[((long long)r << p.lk) + k0 + c] : czero<T>();
        }
        __syncthreads();
        for (int kk = 0; kk < kt; kk++) {
            T a[RM], b[RN];
#pragma unroll
            for (int i = 0; i < RM; i++) a[i] = As[kk][ty * RM + i];
#pragma unroll
            for (int j = 0; j < RN; j++) b[j] = Bs[kk][tx + j * NTX];
#pragma unroll
            for (int i = 0; i < RM; i++)
#pragma unroll
                for (int j = 0; j < RN; j++) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    const long long cb = scatter_bits(bat, p.pos_bat, p.lbat);
    long long offn[RN];
#pragma unroll
    for (int j = 0; j < RN; j++) offn[j] = scatter_bits(n0 + tx + j * NTX, p.pos_n, p.ln);
#pragma unroll
    for (int i = 0; i < RM; i++) {
        const int r = ty * RM + i;
        if (r >= mrows) continue;
        const long long offm = cb + scatter_bits(m0 + r, p.pos_m, p.lm);
#pragma unroll
        for (int j = 0; j < RN; j++)
            if (tx + j * NTX < ncols) store_c_t<T>(p, v, offm + offn[j], acc[i][j]);
    }
}

// ---------------------------------------------------------------- leaves

struct MatDesc {
    const double2 *src;  // full leaf tensor, data index = sum_t value(leg t) << t
    void *dst;           // [code][2^nd] in the consumer's layout and format
    int fmt;             // OutFmt (complex64 leaves only; complex128 when T = double2)
    float scale;         // multiplier (split fp16 range scaling)
    int nd;              // destination bits
    int ncode_bits;      // sliced legs of the leaf
    int8_t dst_leg[kMaxBits];  // destination bit -> source leg position
    int8_t sl_leg[8];          // code bit u -> source leg position
};

// grid.y = leaf; threads over (code, element).
template <typename T>
__global__ void materialize(const MatDesc *descs) {
    const MatDesc d = descs[blockIdx.y];
    const long long total = 1LL << (d.nd + d.ncode_bits);
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long code = g >> d.nd, e = g & ((1LL << d.nd) - 1);
        long long src = 0;
        for (int t = 0; t < d.nd; t++) src |= ((e >> t) & 1) << d.dst_leg[t];
        for (int u = 0; u < d.ncode_bits; u++) src |= ((code >> u) & 1) << d.sl_leg[u];
        const double2 x = d.src[src];
        if constexpr (sizeof(T) == sizeof(float2)) {
            const float2 y = make_float2((float)(x.x * d.scale), (float)(x.y * d.scale));
            if (d.fmt == OUT_C64) {
                static_cast<float2 *>(d.dst)[g] = y;
            } else {
                const long long ne = 1LL << d.nd;
                unsigned short *base = static_cast<unsigned short *>(d.dst) + 4 * code * ne;
                store_split(base, ne, e, y, d.fmt == OUT_SPLIT_FP16);
            }
        } else {
            static_cast<T *>(d.dst)[g] = x;
        }
    }
}

// ---------------------------------------------------------------- batch gathers

__device__ __forceinline__ void gather_copy(const GatherDesc &d, long long vp, long long e, long long se) {
    const char *src = d.src + (vp * d.src_plane + se) * d.esize;
    char *dst = d.dst + (vp * d.dst_plane + e) * d.esize;
    if (d.vec_log2 > 0 || d.esize == 16) *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
    else if (d.esize == 8) *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(src);
    else *reinterpret_cast<unsigned short *>(dst) = *reinterpret_cast<const unsigned short *>(src);
}

// grid.y = gather.  Runs of at least 32 chunks: one warp per run decodes the batch and
// selection once and its lanes copy the run's 16-byte chunks; shorter runs: one thread
// per chunk.  The descriptor is staged in shared memory.
__global__ void gather_batches(const GatherDesc *descs, const uint64_t *closed_bits) {
    __shared__ GatherDesc d;
    if (threadIdx.x == 0) d = descs[blockIdx.y];
    __syncthreads();
    const int vl = d.vec_log2;
    const long long per_plane = d.dst_plane >> vl;  // chunks per plane
    if (d.run_log2 >= 5) {
        const int lr = d.run_log2, lane = threadIdx.x & 31;
        const long long runs_plane = per_plane >> lr;
        const long long runs = runs_plane * d.nplanes * d.nver;
        const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
        for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < runs; r += nw) {
            const long long vp = r / runs_plane;
            const long long e0 = (r - vp * runs_plane) << (lr + vl);
            const long long se0 = gather_src(d, e0, closed_bits);
            for (long long c = lane; c < (1LL << lr); c += 32) gather_copy(d, vp, e0 + (c << vl), se0 + (c << vl));
        }
        return;
    }
    const long long total = per_plane * d.nplanes * d.nver;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const long long vp = g / per_plane;
        const long long e = (g - vp * per_plane) << vl;
        gather_copy(d, vp, e, gather_src(d, e, closed_bits));
    }
}

// ---------------------------------------------------------------- calibration

// *absmax_bits = max(*absmax_bits, max |re|, |im| over the n elements of one version of a
// tensor stored in format fmt (split formats: planes 0 and 2, the hi parts).  Non-negative
// floats compare as integers.
__global__ void absmax_kernel(const void *data, long long n, int fmt, int *absmax_bits) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (fmt == OUT_C64) {
            const float2 x = static_cast<const float2 *>(data)[i];
            m = fmaxf(m, fmaxf(fabsf(x.x), fabsf(x.y)));
        } else {
            const __nv_bfloat16 *h = static_cast<const __nv_bfloat16 *>(data);
            m = fmaxf(m, fmaxf(fabsf(__bfloat162float(h[i])), fabsf(__bfloat162float(h[2 * n + i]))));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(absmax_bits, __float_as_int(m));
}

// ---------------------------------------------------------------- slice sum

// out[e] = sum over explicit root versions v (in order) and over the 2^nfree patterns f
// of the sliced legs carried as layout bits (ascending) of root_v[(f << nout) | e], FP64.
// complex64 inputs are widened with integer operations (exact), which leaves the FP64
// pipe to the additions.
__device__ __forceinline__ double slice_widen(float x) { return tn_widen(x); }
__device__ __forceinline__ double slice_widen(double x) { return x; }

template <typename T>
__global__ void slice_sum(const void *const *ptr, long long nver, int nfree, int nout, double2 *out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (1LL << nout)) return;
    double re = 0.0, im = 0.0;
    const long long nf = 1LL << nfree;
    for (long long v = 0; v < nver; v++) {
        const T *r = static_cast<const T *>(ptr[v]) + e;
        long long f = 0;
        // loads issued four at a time; the additions stay in slice order
        for (; f + 4 <= nf; f += 4) {
            const T x0 = r[(f + 0) << nout], x1 = r[(f + 1) << nout], x2 = r[(f + 2) << nout], x3 = r[(f + 3) << nout];
            re = __dadd_rn(re, slice_widen(x0.x));
            im = __dadd_rn(im, slice_widen(x0.y));
            re = __dadd_rn(re, slice_widen(x1.x));
            im = __dadd_rn(im, slice_widen(x1.y));
            re = __dadd_rn(re, slice_widen(x2.x));
            im = __dadd_rn(im, slice_widen(x2.y));
            re = __dadd_rn(re, slice_widen(x3.x));
            im = __dadd_rn(im, slice_widen(x3.y));
        }
        for (; f < nf; f++) {
            const T x = r[f << nout];
            re = __dadd_rn(re, slice_widen(x.x));
            im = __dadd_rn(im, slice_widen(x.y));
        }
    }
    out[e] = make_double2(re, im);
}

// ---------------------------------------------------------------- root product + slice sum

// The batch, row and column bits of C position pos under the row-kernel parameters p
// (pos_* give each bit's C position; positions no bit maps to contribute nothing).
__device__ __forceinline__ void root_split(const GemmParams &p, long long pos, long long &bat, long long &m, int &n) {
    bat = 0;
    m = 0;
    n = 0;
    for (int i = 0; i < p.lbat; i++) bat |= ((pos >> p.pos_bat[i]) & 1LL) << i;
    for (int i = 0; i < p.lm; i++) m |= ((pos >> p.pos_m[i]) & 1LL) << i;
    for (int i = 0; i < p.ln; i++) n |= (int)((pos >> p.pos_n[i]) & 1LL) << i;
}

// The value cgemm_row_one stores for output (v, bat, m, n), before the store: the same
// operand rows (gathered ones read in place), k order and multiply-add operand order.
template <typename T>
__device__ __forceinline__ T root_value(const GemmParams &p, long long v, long long bat, long long m, int n) {
    const T *A, *B;
    if (p.gA) {
        const long long e = ((bat << p.lm) | m) << p.lk;
        A = reinterpret_cast<const T *>(p.gA->src) + gather_src_warp(*p.gA, e, p.gA->pos_beta[p.gA->lb - 1], p.closed_bits);
    } else {
        A = static_cast<const T *>(p.ptrA[v]) + (((bat << p.lm) | m) << p.lk);
    }
    if (p.gB) {
        const long long e = bat << (p.ln + p.lk);
        B = reinterpret_cast<const T *>(p.gB->src) + gather_src_warp(*p.gB, e, p.gB->pos_beta[p.gB->lb - 1], p.closed_bits);
    } else {
        B = static_cast<const T *>(p.ptrB[v]) + (bat << (p.ln + p.lk));
    }
    B += (long long)n << p.lk;
    const int K = 1 << p.lk;
    T acc = czero<T>();
    if (p.swapped) {
        for (int k = 0; k < K; k++) acc = cfma(__ldg(&B[k]), A[k], acc);
    } else {
        for (int k = 0; k < K; k++) acc = cfma(A[k], __ldg(&B[k]), acc);
    }
    return acc;
}

// What store_c_t applies before storing: the output scale for complex64, nothing for
// complex128.
__device__ __forceinline__ float2 root_scaled(const GemmParams &p, float2 x) {
    x.x *= p.out_scale;
    x.y *= p.out_scale;
    return x;
}
__device__ __forceinline__ double2 root_scaled(const GemmParams &, double2 x) { return x; }

constexpr int kRootTabBytes = 3;  // free patterns of up to 24 bits

// The root step fused with the slice sum: out[e] = sum over explicit root versions v (in
// order) and free patterns f (ascending) of the root product's value at C position
// (f << nout) | e, p being the root step's row-kernel parameters.  Each value is formed
// as the row kernel forms it and widened and added in FP64 in slice_sum's order, so out is
// bit-identical to the row kernel followed by slice_sum, and the root's 2^(nout + nfree)
// values never pass through memory.  The host checks that p's batch, row and column bits
// cover the positions [0, nout + nfree) once each, so every (bat, m, n) below is in range.
template <typename T>
__global__ void __launch_bounds__(256) root_slice_sum(GemmParams p, int nfree, int nout, double2 *out) {
    // byte tables: t*[j][b] are the batch, row and column bits of position (b << 8j) << nout
    __shared__ long long tbat[kRootTabBytes][256], tm[kRootTabBytes][256];
    __shared__ int tn[kRootTabBytes][256];
    const int nbytes = (nfree + 7) >> 3;
    for (int i = threadIdx.x; i < nbytes * 256; i += blockDim.x) {
        const int j = i >> 8;
        long long b, m;
        int n;
        root_split(p, ((long long)(i & 255) << (8 * j)) << nout, b, m, n);
        tbat[j][i & 255] = b;
        tm[j][i & 255] = m;
        tn[j][i & 255] = n;
    }
    __syncthreads();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (1LL << nout)) return;
    long long be, me;
    int ne;
    root_split(p, e, be, me, ne);
    const long long nf = 1LL << nfree;
    double re = 0.0, im = 0.0;
    for (long long v = 0; v < p.nver; v++) {
        for (long long f = 0; f < nf; f++) {
            long long bat = be, m = me;
            int n = ne;
            for (int j = 0; j < nbytes; j++) {
                const int b = (int)((f >> (8 * j)) & 255);
                bat |= tbat[j][b];
                m |= tm[j][b];
                n |= tn[j][b];
            }
            const T x = root_scaled(p, root_value<T>(p, v, bat, m, n));
            re = __dadd_rn(re, slice_widen(x.x));
            im = __dadd_rn(im, slice_widen(x.y));
        }
    }
    out[e] = make_double2(re, im);
}

// ---------------------------------------------------------------- sampling job

// acc[e] += x[e] in FP64 for e < n: a sampling job adds each slice chunk's sum over its
// slices (Sec. I.C step 1) to the running total of the same batches, chunk after chunk,
// so every amplitude is summed in one fixed order.
__global__ void accumulate_amps(double2 *acc, const double2 *x, long long n) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double2 a = acc[e], b = x[e];
        acc[e] = make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
    }
}

// ---------------------------------------------------------------- verification XEB

// The amplitude of each of nb bitstrings from its batch: out[t] = amps[(t << n_open) | idx[t]].
__global__ void pick_amplitudes(const double2 *amps, int n_open, const int32_t *idx, long long nb, double2 *out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nb) out[t] = amps[(t << n_open) | idx[t]];
}

// FP64 sum of |a_i|^2 = re*re + im*im (rounded products, no fused multiply-add) over n
// values in a fixed order: thread j of block b sums i = b*256 + j, then every stride of
// kNormGrid*256, in turn; each block halves its 256 partials pairwise into partial[b].
// norm_total then halves the kNormGrid partials the same way.
constexpr int kNormGrid = 256;
__global__ void __launch_bounds__(256) sum_norms(const double2 *a, long long n, double *partial) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)kNormGrid * 256)
        acc = __dadd_rn(acc, __dadd_rn(__dmul_rn(a[i].x, a[i].x), __dmul_rn(a[i].y, a[i].y)));
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}
__global__ void __launch_bounds__(256) norm_total(const double *partial, double *out) {
    __shared__ double sh[kNormGrid];
    sh[threadIdx.x] = partial[threadIdx.x];
    __syncthreads();
    for (int h = kNormGrid / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// ---------------------------------------------------------------- top-N selection (XEB spoofing)

// key[i] = the bit pattern of p_i = re*re + im*im in FP64 (rounded products, no fused
// multiply-add): non-negative doubles order like their bit patterns.
__global__ void spoof_keys(const double2 *a, long long n, unsigned long long *key) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double p = __dadd_rn(__dmul_rn(a[i].x, a[i].x), __dmul_rn(a[i].y, a[i].y));
        key[i] = (unsigned long long)__double_as_longlong(p);
    }
}

// Histogram of the 8-bit digit at `shift` over the keys whose bits above it equal `prefix`
// (under `mask`): one shared histogram per block, added to hist[256].
__global__ void __launch_bounds__(256) digit_hist(const unsigned long long *key, long long n, unsigned long long mask,
                                                  unsigned long long prefix, int shift, unsigned int *hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

constexpr int kSelBlock = 1024;  // keys per selection block (one per thread)

// Exclusive rank of this thread's flag among the block's flags, and the block's total.
__device__ __forceinline__ unsigned int block_rank(bool f, unsigned int *warp_tot, unsigned int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int b = __ballot_sync(0xffffffffu, f);
    const unsigned int in_warp = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(b);
    __syncthreads();
    unsigned int before = 0;
    total = 0;
    for (int w = 0; w < kSelBlock / 32; w++) {
        if (w < warp) before += warp_tot[w];
        total += warp_tot[w];
    }
    __syncthreads();  // warp_tot is reused by the next call
    return before + in_warp;
}

// Per block of kSelBlock consecutive keys: how many exceed the threshold and how many equal it.
__global__ void __launch_bounds__(kSelBlock) sel_counts(const unsigned long long *key, long long n,
                                                        unsigned long long thr, unsigned int *gt, unsigned int *eq) {
    __shared__ unsigned int wt[kSelBlock / 32];
    const long long i = (long long)blockIdx.x * kSelBlock + threadIdx.x;
    const unsigned long long k = i < n ? key[i] : 0ull;
    unsigned int tg, te;
    block_rank(i < n && k > thr, wt, tg);
    block_rank(i < n && k == thr, wt, te);
    if (threadIdx.x == 0) {
        gt[blockIdx.x] = tg;
        eq[blockIdx.x] = te;
    }
}

// In-place exclusive prefix sums of the per-block counts, in one block, chunk by chunk.
__global__ void __launch_bounds__(kSelBlock) sel_scan(unsigned int *gt, unsigned int *eq, int nb) {
    __shared__ unsigned int wg[kSelBlock / 32], we[kSelBlock / 32];
    unsigned int carry_g = 0, carry_e = 0;
    for (int c = 0; c < nb; c += kSelBlock) {
        const int j = c + (int)threadIdx.x;
        const unsigned int g = j < nb ? gt[j] : 0u, e = j < nb ? eq[j] : 0u;
        // block-wide exclusive sums of g and e by warp scans (shuffles) of the counts
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        unsigned int sg = g, se = e;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int yg = __shfl_up_sync(0xffffffffu, sg, o), ye = __shfl_up_sync(0xffffffffu, se, o);
            if (lane >= o) {
                sg += yg;
                se += ye;
            }
        }
        if (lane == 31) {
            wg[warp] = sg;
            we[warp] = se;
        }
        __syncthreads();
        unsigned int bg = 0, be = 0, tg = 0, te = 0;
        for (int w = 0; w < kSelBlock / 32; w++) {
            if (w < warp) {
                bg += wg[w];
                be += we[w];
            }
            tg += wg[w];
            te += we[w];
        }
        if (j < nb) {
            gt[j] = carry_g + bg + sg - g;
            eq[j] = carry_e + be + se - e;
        }
        carry_g += tg;
        carry_e += te;
        __syncthreads();  // wg / we are rewritten by the next chunk
    }
}

// The open qubits of a batch: bit r of an in-batch index is qubit q[r].
struct OpenQubits {
    int8_t q[64];
    int n;
};

// Write the selected positions in ascending order: key > thr, or key == thr among the
// first `need` equal ones (by position).  Position i goes out as the bitstring
// base | (bit r of i at qubit open.q[r]) with its p_i.
__global__ void __launch_bounds__(kSelBlock) sel_write(const unsigned long long *key, long long n,
                                                       unsigned long long thr, long long need,
                                                       const unsigned int *gt_off, const unsigned int *eq_off,
                                                       unsigned long long base, OpenQubits open,
                                                       unsigned long long *bits, double *prob) {
    __shared__ unsigned int wt[kSelBlock / 32];
    const long long i = (long long)blockIdx.x * kSelBlock + threadIdx.x;
    const unsigned long long k = i < n ? key[i] : 0ull;
    const bool g = i < n && k > thr, e = i < n && k == thr;
    unsigned int t;
    const unsigned int lg = block_rank(g, wt, t);
    const unsigned int le = block_rank(e, wt, t);
    const long long eq_before = (long long)eq_off[blockIdx.x] + le;
    if (g || (e && eq_before < need)) {
        const long long pos = (long long)gt_off[blockIdx.x] + lg + (eq_before < need ? eq_before : need);
        unsigned long long b = base;
        for (int r = 0; r < open.n; r++) b |= (unsigned long long)((i >> r) & 1) << open.q[r];
        bits[pos] = b;
        if (prob) prob[pos] = __longlong_as_double((long long)k);
    }
}

// ---------------------------------------------------------------- Philox

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
// multiplications with key bumps by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
    const uint64_t w = ((uint64_t)hi << 32) | lo;
    return __dmul_rn((double)(w >> 11), 1.0 / 9007199254740992.0);
}

__global__ void draw_batches(uint64_t seed, uint64_t t0, long long T, int b_bits, uint64_t *j) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint64_t tt = t0 + (uint64_t)t;
    const uint4 o = philox4x32_10(make_uint4((uint32_t)tt, (uint32_t)(tt >> 32), 0u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const uint64_t w = ((uint64_t)o.y << 32) | o.x;
    j[t] = b_bits >= 64 ? w : (w & ((1ull << b_bits) - 1));
}

struct SampleParams {
    const double *p;      // T*64 probabilities, or null (then amps/F)
    const double2 *amps;  // T*64 amplitudes
    double invF_num;      // F (p = |a|^2 / F)
    long long T;
    int b_bits;
    double alpha;
    uint64_t seed, t0;
    uint8_t *accept;
    int32_t *pick;
    double *eps;          // optional: max(0, p_j - alpha/N_B)
    const uint64_t *j;    // optional: batch patterns (for bitstrings)
    uint64_t *bits;       // optional: assembled bitstrings
    int n_open, n_closed;
    int8_t open_q[16];
    int8_t closed_q[64];
};

// One warp per batch (Sec. II.A steps 2-3); lane l holds p_{2l}, p_{2l+1}.
__global__ void sampler(SampleParams sp) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= sp.T) return;
    double p0, p1;
    if (sp.p) {
        p0 = sp.p[warp * 64 + 2 * lane];
        p1 = sp.p[warp * 64 + 2 * lane + 1];
    } else {
        const double2 a0 = sp.amps[warp * 64 + 2 * lane], a1 = sp.amps[warp * 64 + 2 * lane + 1];
        p0 = __ddiv_rn(__dadd_rn(__dmul_rn(a0.x, a0.x), __dmul_rn(a0.y, a0.y)), sp.invF_num);
        p1 = __ddiv_rn(__dadd_rn(__dmul_rn(a1.x, a1.x), __dmul_rn(a1.y, a1.y)), sp.invF_num);
    }
    double x = __dadd_rn(p0, p1);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x = __dadd_rn(y, x);
    }
    const double pj = __shfl_sync(0xffffffffu, x, 31);
    double excl = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) excl = 0.0;
    const uint64_t t = sp.t0 + (uint64_t)warp;
    const uint2 key = make_uint2((uint32_t)sp.seed, (uint32_t)(sp.seed >> 32));
    const uint4 o0 = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 0u, 0u), key);
    const uint4 o1 = philox4x32_10(make_uint4((uint32_t)t, (uint32_t)(t >> 32), 1u, 0u), key);
    const double u = u53(o0.z, o0.w), v = u53(o1.x, o1.y);
    const double NB = ldexp(1.0, sp.b_bits);
    const bool acc = __dmul_rn(u, sp.alpha) < __dmul_rn(pj, NB);
    const double tau = __dmul_rn(v, pj);
    const double c0 = __dadd_rn(excl, p0), c1 = x;
    const bool h0 = c0 > tau, h1 = c1 > tau;
    const unsigned hit = __ballot_sync(0xffffffffu, h0 || h1);
    int pick;
    if (hit) {
        const int L = __ffs(hit) - 1;
        const bool l0 = __shfl_sync(0xffffffffu, h0, L);
        pick = l0 ? 2 * L : 2 * L + 1;
    } else {
        const unsigned nz = __ballot_sync(0xffffffffu, p0 > 0.0 || p1 > 0.0);
        if (nz) {
            const int L = 31 - __clz(nz);
            const bool z1 = __shfl_sync(0xffffffffu, p1 > 0.0, L);
            pick = z1 ? 2 * L + 1 : 2 * L;
        } else {
            pick = 63;
        }
    }
    if (lane == 0) {
        sp.accept[warp] = acc ? 1 : 0;
        sp.pick[warp] = pick;
        if (sp.eps) sp.eps[warp] = fmax(__dadd_rn(pj, -sp.alpha / NB), 0.0);
        if (sp.bits) {
            const uint64_t jj = sp.j[warp];
            uint64_t b = 0;
            for (int r = 0; r < sp.n_open; r++) b |= (uint64_t)((pick >> r) & 1) << sp.open_q[r];
            for (int c = 0; c < sp.n_closed; c++) b |= ((jj >> c) & 1ull) << sp.closed_q[c];
            sp.bits[warp] = b;
        }
    }
}

// ---------------------------------------------------------------- slice cut

// Alg. 1 steps 4-5 for 2^k <= 4096 norms in one block: bitonic sort of (R desc, i asc)
// in shared memory, then a sequential FP64 prefix in sorted order.
__global__ void slice_cut(const double *R, int k, double f, int32_t *X, int32_t *n_x, double *F) {
    extern __shared__ unsigned char smem[];
    const int n = 1 << k;
    double *r = reinterpret_cast<double *>(smem);
    int *idx = reinterpret_cast<int *>(r + n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) { r[i] = R[i]; idx[i] = i; }
    __syncthreads();
    for (int size = 2; size <= n; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    // "before(a, b)": a precedes b in (R descending, index ascending) order
                    const bool a_first = r[i] > r[j] || (r[i] == r[j] && idx[i] < idx[j]);
                    const bool up = (i & size) == 0;
                    if (up != a_first) {
                        const double tr = r[i]; r[i] = r[j]; r[j] = tr;
                        const int ti = idx[i]; idx[i] = idx[j]; idx[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        double acc = 0.0;
        int cnt = n;
        for (int t = 0; t < n; t++) {
            acc = __dadd_rn(acc, r[t]);
            if (acc >= f) { cnt = t + 1; break; }
        }
        *n_x = cnt;
        *F = acc;
    }
    __syncthreads();
    const int cnt = *n_x;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) X[t] = idx[t];
}

}  // namespace tnk
