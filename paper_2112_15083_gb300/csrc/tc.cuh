// tcgen05 split-precision complex GEMM (sm_103a) for the contraction steps.
//
// C[bat][m][n] = sum_k A[bat][m][k] * B[bat][n][k] with A and B stored as four planes
// (re_hi, re_lo, im_hi, im_lo) of bf16 or fp16, plane-major: plane p of batch b is the
// row-major [rows][K] matrix at plane index p * BAT + b.  With x = hi + lo the complex
// product keeps hi*hi + hi*lo + lo*hi of each real product:
//   Cr = Ar Br - Ai Bi,  Ci = Ar Bi + Ai Br,
// i.e. 12 tensor-core MMAs per K slice accumulated in FP32 in two TMEM accumulators
// (Cr, Ci); the subtracted products use the descriptor's negate-A bit.
//
// One CTA computes a 128 x BN tile: warp 0 / lane 0 streams the 8 operand plane tiles
// of each 32-wide K slice with 4-D TMA (64-byte swizzle) into a ring of stages, warp 1 /
// lane 0 issues the MMAs and releases ring slots with tcgen05.commit, and eight epilogue
// warps read the accumulators back with tcgen05.ld (warp w owns TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31, i.e. tile rows, and half of the columns) and store in the
// consumer's format through the bit-scatter epilogue.
// Every mbarrier wait is bounded: on timeout the CTA sets *err, stops, waits (bounded)
// for work it already issued, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "kernels.cuh"

namespace tnk {

constexpr int kTcBM = 128;
constexpr int kTcBK = 32;      // K elements per ring slot (64 bytes per row: 64B swizzle)

// An operand read in place from its stored form instead of a per-batch gathered copy.
// The stored form is the read layout [K][rows][non-beta batch bits] with the operand's
// closed legs on top; a tile of batch `bat` reads plane coordinate (non-beta bits of bat)
// | (the batch pattern's bits q[0..nq) packed) << nnb, the pattern being the group's
// closed_bits[beta index of bat].
struct TcGather {
    const uint64_t *closed;  // null: the operand is read as laid out (no gather)
    uint32_t beta_mask;      // bits of bat that are beta (batch-index) bits
    int8_t beta_t[24];       // for such bit i: which bit of the batch index it is
    int nnb;                 // non-beta bits of bat
    int nq;
    int8_t q[32];            // closed positions of the pattern bits, lowest first
};

// The stored block a batch pattern selects: its bits at the closed positions q[].
__device__ __forceinline__ int tc_gather_sel(const TcGather &g, uint64_t pat) {
    int sel = 0;
    for (int t = 0; t < g.nq; t++) sel |= (int)((pat >> g.q[t]) & 1ull) << t;
    return sel;
}

__device__ __forceinline__ int tc_gather_plane(const TcGather &g, int lbat, int bat) {
    int beta = 0, nonb = 0, j = 0;
    for (int i = 0; i < lbat; i++) {
        const int bit = (bat >> i) & 1;
        if ((g.beta_mask >> i) & 1) beta |= bit << g.beta_t[i];
        else nonb |= bit << j++;
    }
    return nonb | (tc_gather_sel(g, g.closed[beta]) << g.nnb);
}

// The batch index whose beta bits are `beta` and whose other bits are `nonb` (lowest first).
__device__ __forceinline__ int tc_compose_bat(const TcGather &g, int lbat, int nonb, int beta) {
    int bat = 0, j = 0;
    for (int i = 0; i < lbat; i++) {
        const int bit = ((g.beta_mask >> i) & 1) ? (beta >> g.beta_t[i]) & 1 : (nonb >> j++) & 1;
        bat |= bit << i;
    }
    return bat;
}

// Stacked tiles.  The batches of a group whose patterns select the same stored block of
// the in-place operand A multiply the same A matrix; a stacked tile takes up to S of them
// (S = BN / N) and puts their B rows side by side in its BN columns, so the A panel is
// loaded once for S batches and one MMA of BN columns serves them all.  The stack list is
// built on the device per group (tc_stack_build): word 0 the number of stacks, then S + 1
// words per stack: the selected block, then S batch indices (beta), -1 in unused slots
// (the valid ones first).
constexpr int kTcMaxStack = 4;

// Sorts the group's T = 2^nbeta batch indices by (selected block, beta) with a bitonic
// sort in shared memory (deterministic), then cuts each block's run into stacks of S.
// One block of 1024 threads; dynamic shared memory 8 T bytes.
__global__ void __launch_bounds__(1024) tc_stack_build(TcGather g, int nbeta, int S, int *out) {
    extern __shared__ unsigned long long keys[];
    __shared__ int scan[1024];
    const int T = 1 << nbeta, nt = blockDim.x, tid = threadIdx.x;
    for (int b = tid; b < T; b += nt)
        keys[b] = ((unsigned long long)(unsigned)tc_gather_sel(g, g.closed[b]) << 32) | (unsigned)b;
    for (int i = tid; i < T * (S + 1); i += nt) out[1 + i] = -1;
    __syncthreads();
    for (int k = 2; k <= T; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < T; i += nt) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = keys[i], c = keys[l];
                    if ((a > c) == ((i & k) == 0)) {
                        keys[i] = c;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // thread tid walks positions [lo, hi) of the sorted list; a run starts where the block
    // changes, and a stack at every S-th position of a run
    const int E = (T + nt - 1) / nt, lo = min(T, tid * E), hi = min(T, lo + E);
    auto head = [&](int i) { return i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32); };
    int last = -1;
    for (int i = lo; i < hi; i++)
        if (head(i)) last = i;
    scan[tid] = last;  // inclusive max-scan: the last run start at or before the chunk's end
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        const int v = tid >= d ? scan[tid - d] : -1;
        __syncthreads();
        scan[tid] = max(scan[tid], v);
        __syncthreads();
    }
    const int run0 = tid > 0 ? scan[tid - 1] : -1;
    __syncthreads();
    int starts = 0;
    last = run0;
    for (int i = lo; i < hi; i++) {
        if (head(i)) last = i;
        starts += (i - last) % S == 0;
    }
    scan[tid] = starts;  // inclusive sum-scan of the stack starts
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        const int v = tid >= d ? scan[tid - d] : 0;
        __syncthreads();
        scan[tid] += v;
        __syncthreads();
    }
    int id = scan[tid] - starts - 1;  // stacks started before this chunk, minus one
    last = run0;
    for (int i = lo; i < hi; i++) {
        if (head(i)) last = i;
        const int pos = (i - last) % S;
        int *e = out + 1 + (id + (pos == 0)) * (S + 1);
        if (pos == 0) {
            id++;
            e[0] = (int)(keys[i] >> 32);
        }
        e[1 + pos] = (int)(keys[i] & 0xffffffffu);
    }
    if (tid == nt - 1) out[0] = scan[tid];
}

struct TcParams {
    void *C;                 // output base (version 0); version v at C + 8 * v * c_plane bytes
    long long c_plane;       // elements per version (= split plane stride)
    const int *vidx;         // [v]: A version index, [nver + v]: B version index
    int nver;                // explicit versions of C (power of two not required)
    int fold;                // 0: versions are tiles; 1: versions folded into M; 2: into N
    int lm, ln, lk, lbat;
    int out_fmt;
    int in_fp16;             // operands are fp16 (else bf16)
    float out_scale;         // multiply results by this before storing
    int *err;                // set to 1 if a bounded wait gives up
    int group_m;             // m tiles per raster group (>= 1): see tc_tile
    long long stall_cycles;  // > 0 (tests only): the MMA warp first waits this long on a
                             // barrier nothing arrives on, so the bounded-wait path runs
    TcGather ga, gb;         // operands read in place through their batch gather
    const int *stack;        // non-null: stacked tiles over this stack list (tc_stack_build)
    int stack_S;             // batches per stacked tile (BN >> ln)
    int8_t pos_bat[kMaxBits], pos_m[kMaxBits], pos_n[kMaxBits];
};

// Tile t of a launch: (batch, version) outermost; inside, groups of group_m m tiles are
// walked n tile by n tile with the m tiles of the group fastest, so the CTAs running
// together share a few operand panels of both A and B in L2 (with group_m = 1 this is
// the plain n-fastest order).
struct TcTile {
    int tn_i, tm_i, bat;
    long long v;
};

// Stacked tile t: m tiles fastest, then stacks (sorted by block: the stacks of one block
// run back to back and share its panels in L2), then the non-beta batch bits, then version.
struct TcStackTile {
    int tm_i, stack, nonb;
    long long v;
};
__device__ __forceinline__ TcStackTile tc_stack_tile(long long t, long long tiles_m, int n_stacks, int nnb) {
    TcStackTile r;
    r.tm_i = (int)(t % tiles_m);
    long long q = t / tiles_m;
    r.stack = (int)(q % n_stacks);
    q /= n_stacks;
    r.nonb = (int)(q & ((1LL << nnb) - 1));
    r.v = q >> nnb;
    return r;
}

__device__ __forceinline__ TcTile tc_tile(long long t, long long tiles_m, long long tiles_n, int lbat, int group_m) {
    const long long per_bat = tiles_m * tiles_n;
    const long long bv = t / per_bat, tl = t - bv * per_bat;
    TcTile r;
    r.bat = (int)(bv & ((1LL << lbat) - 1));
    r.v = bv >> lbat;
    const long long gsz = (long long)group_m * tiles_n;
    const long long g = tl / gsz, rr = tl - g * gsz;
    const long long gm = min((long long)group_m, tiles_m - g * group_m);
    r.tn_i = (int)(rr / gm);
    r.tm_i = (int)(g * group_m + rr % gm);
    return r;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile, 64-byte swizzle, 8-row groups 512 B
// apart (rows are 64 bytes), start address advanced by 32 B per 16-element K step.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)4 << 61;            // 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A/B = BF16 (1) or F16 (0), K-major both,
// N >> 3 at bit 17, M >> 4 at bit 24, optional negation of A.
__device__ __forceinline__ uint32_t idesc_f16(int n, bool fp16, bool neg_a) {
    uint32_t ab = fp16 ? 0u : 1u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTcBM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Both accumulators' 16 columns (Cr, Ci) with one wait for the two loads.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float *va, float *vb) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(r[16 + i]);
    }
}

template <int BN, int STAGES>
struct TcSmem {
    static constexpr int kAPlane = kTcBM * kTcBK * 2;  // bytes per A plane tile
    static constexpr int kBPlane = BN * kTcBK * 2;
    static constexpr int kStage = 4 * kAPlane + 4 * kBPlane;
    static constexpr int kBytes = STAGES * kStage + 1024 /*barriers*/ + 1024 /*alignment*/;
};

constexpr int kTcEpiWarps = 8;   // two per TMEM lane quarter, each owning half the tile's columns
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;  // warp 0: TMA, warp 1: MMA, warps 2-9: epilogue

// Persistent kernel: CTA c processes tiles c, c + gridDim.x, ...  Tile order: N tiles
// fastest, then M tiles, then batch, then explicit version (CTAs running together share
// the A row panel).  Operand maps are 4-D: [version][4 * BAT planes][rows][K].
// TMEM holds two accumulator pairs (Cr | Ci for BN columns each) so the epilogue of
// one tile overlaps the MMAs of the next.
template <int BN, int STAGES>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_cgemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
    using L = TcSmem<BN, STAGES>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *ctl = smem + STAGES * L::kStage;
    uint64_t *full = reinterpret_cast<uint64_t *>(ctl);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;  // [2]: MMA -> epilogue
    uint64_t *acc_empty = acc_full + 2;   // [2]: epilogue -> MMA
    uint64_t *never = acc_empty + 2;      // test stall: initialised, never arrived on
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(never + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *slot_cols = abort_flag + 1;  // [STAGES]: a stacked tile's MMA width

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Tiles: (n tile, m tile, batch, version) without folding.  With folding the rows
    // (fold 1) or columns (fold 2) of all versions form one axis: versions are stacked,
    // 128/M (or BN/N) per tile, and the operand's map box spans that many versions.
    const int ltm = min(p.lm, 7), ltn = min(p.ln, __ffs(BN) - 1);
    const int vm = p.fold == 1 ? (kTcBM >> p.lm) : 1;  // versions per m tile
    const int vn = p.fold == 2 ? (BN >> p.ln) : 1;      // versions per n tile
    const long long tiles_m = p.fold == 1 ? (p.nver + vm - 1) / vm : (1LL << (p.lm - ltm));
    const long long tiles_n = p.fold == 2 ? (p.nver + vn - 1) / vn : (1LL << (p.ln - ltn));
    const long long tiles_v = p.fold ? 1 : p.nver;
    const long long per_bat = tiles_m * tiles_n;
    // stacked: (version, non-beta bits, stack, m tile); the host guarantees one n tile
    const bool stk = p.stack != nullptr;
    const int S = p.stack_S, n_stacks = stk ? p.stack[0] : 0;
    const long long ntiles =
        stk ? tiles_m * n_stacks * (1LL << p.ga.nnb) * tiles_v : per_bat * (1LL << p.lbat) * tiles_v;
    const int BAT = 1 << p.lbat;
    const int K = 1 << p.lk;
    const int nkb = (K + kTcBK - 1) / kTcBK;
    constexpr uint32_t kCols = 4 * BN;  // two accumulator pairs
    const long long kLimit = 4000000000LL;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kTcEpiWarps);  // one arrive per epilogue warp
        }
        mbar_init(smem_u32(never), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    long long issued = 0;  // producer: ring slots issued
    if (warp == 0) {
        if (lane == 0) {
            long long slot = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok && !stk; t += gridDim.x) {
                const TcTile tt = tc_tile(t, tiles_m, tiles_n, p.lbat, p.group_m);
                const int tn_i = tt.tn_i, tm_i = tt.tm_i, bat = tt.bat, v = (int)tt.v;
                const int ia = p.fold == 1 ? p.vidx[0] + tm_i * vm : p.vidx[p.fold == 2 ? 0 : v];
                const int ib = p.fold == 2 ? p.vidx[p.nver] + tn_i * vn : p.vidx[p.nver + (p.fold == 1 ? 0 : v)];
                const int rowA = p.fold == 1 ? 0 : tm_i * kTcBM, rowB = p.fold == 2 ? 0 : tn_i * BN;
                // plane coordinates: plane pl of batch bat, or of its stored pattern block
                const int pza = p.ga.closed ? tc_gather_plane(p.ga, p.lbat, bat) : bat;
                const int pzb = p.gb.closed ? tc_gather_plane(p.gb, p.lbat, bat) : bat;
                const int sza = p.ga.closed ? 1 << (p.ga.nnb + p.ga.nq) : BAT;
                const int szb = p.gb.closed ? 1 << (p.gb.nnb + p.gb.nq) : BAT;
                for (int kb = 0; kb < nkb; kb++, slot++) {
                    const int s = (int)(slot % STAGES);
                    if (slot >= STAGES &&
                        !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((slot / STAGES) & 1) ^ 1), abort_flag, kLimit)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, L::kStage);
                    unsigned char *st = smem + s * L::kStage;
                    for (int pl = 0; pl < 4; pl++) {
                        tma_load_4d(smem_u32(st + pl * L::kAPlane), &tmA, kb * kTcBK, rowA, pl * sza + pza, ia, fb);
                        tma_load_4d(smem_u32(st + 4 * L::kAPlane + pl * L::kBPlane), &tmB, kb * kTcBK, rowB,
                                    pl * szb + pzb, ib, fb);
                    }
                    issued = slot + 1;
                }
            }
            // stacked tiles: one A panel, then one (1 << ln)-row B box per batch of the stack
            // (its valid slots come first); the next tile's stack entry is loaded while this
            // tile's slots are issued, and every slot tells the MMA thread its width
            auto entry = [&](long long t) {
                return p.stack + 1 + (long long)tc_stack_tile(t, tiles_m, n_stacks, p.ga.nnb).stack * (S + 1);
            };
            int nx[kTcMaxStack + 1];
            if (stk && blockIdx.x < ntiles) {
                const int *sb = entry(blockIdx.x);
#pragma unroll
                for (int j = 0; j <= kTcMaxStack; j++) nx[j] = j <= S ? sb[j] : -1;
            }
            for (long long t = blockIdx.x; t < ntiles && ok && stk; t += gridDim.x) {
                int e[kTcMaxStack + 1];
#pragma unroll
                for (int j = 0; j <= kTcMaxStack; j++) e[j] = nx[j];
                if (t + gridDim.x < ntiles) {
                    const int *sb = entry(t + gridDim.x);
#pragma unroll
                    for (int j = 0; j <= kTcMaxStack; j++) nx[j] = j <= S ? sb[j] : -1;
                }
                const TcStackTile tt = tc_stack_tile(t, tiles_m, n_stacks, p.ga.nnb);
                const int pza = tt.nonb | (e[0] << p.ga.nnb);  // the block the stack selects
                const int sza = 1 << (p.ga.nnb + p.ga.nq);
                int pzb[kTcMaxStack], nbox = 0;
#pragma unroll
                for (int j = 0; j < kTcMaxStack; j++) {
                    pzb[j] = -1;
                    if (e[1 + j] >= 0) {
                        const int bat = tc_compose_bat(p.ga, p.lbat, tt.nonb, e[1 + j]);
                        pzb[j] = p.gb.closed ? tc_gather_plane(p.gb, p.lbat, bat) : bat;
                        nbox++;
                    }
                }
                const int ia = p.vidx[tt.v], ib = p.vidx[p.nver + tt.v];
                const int rowA = tt.tm_i * kTcBM;
                const int szb = p.gb.closed ? 1 << (p.gb.nnb + p.gb.nq) : BAT;
                const int bbox = (kTcBK * 2) << p.ln;  // bytes per B box
                for (int kb = 0; kb < nkb; kb++, slot++) {
                    const int s = (int)(slot % STAGES);
                    if (slot >= STAGES &&
                        !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((slot / STAGES) & 1) ^ 1), abort_flag, kLimit)) {
                        ok = false;
                        break;
                    }
                    slot_cols[s] = nbox << p.ln;  // published by the arrive below
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, (uint32_t)(4 * L::kAPlane + 4 * nbox * bbox));
                    unsigned char *st = smem + s * L::kStage;
                    for (int pl = 0; pl < 4; pl++) {
                        tma_load_4d(smem_u32(st + pl * L::kAPlane), &tmA, kb * kTcBK, rowA, pl * sza + pza, ia, fb);
#pragma unroll
                        for (int j = 0; j < kTcMaxStack; j++)
                            if (pzb[j] >= 0)
                                tma_load_4d(smem_u32(st + 4 * L::kAPlane + pl * L::kBPlane + j * bbox), &tmB,
                                            kb * kTcBK, 0, pl * szb + pzb[j], ib, fb);
                    }
                    issued = slot + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // products (A plane, B plane, accumulator 0 = Cr / 1 = Ci, negate A);
            // planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo
            const int8_t pa[12] = {0, 0, 1, 2, 2, 3, 0, 0, 1, 2, 2, 3};
            const int8_t pb[12] = {0, 1, 0, 2, 3, 2, 2, 3, 2, 0, 1, 0};
            const int8_t acc[12] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1};
            const int8_t neg[12] = {0, 0, 0, 1, 1, 1, 0, 0, 0, 0, 0, 0};
            uint32_t id_pos = idesc_f16(BN, p.in_fp16, false), id_neg = idesc_f16(BN, p.in_fp16, true);
            long long slot = 0;
            int it = 0, last_b = -1;
            uint32_t last_par = 0;
            bool ok = true;
            // test hook: a wait that runs out before any MMA is issued
            if (p.stall_cycles > 0) ok = mbar_wait(smem_u32(never), 0u, abort_flag, p.stall_cycles);
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, it++) {
                const int b = it & 1;
                if (it >= 2 &&
                    !mbar_wait(smem_u32(&acc_empty[b]), (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag, kLimit)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dcol = tmem + (uint32_t)(b * 2 * BN);
                for (int kb = 0; kb < nkb; kb++, slot++) {
                    const int s = (int)(slot % STAGES);
                    if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((slot / STAGES) & 1), abort_flag, kLimit)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (stk && kb == 0) {
                        // a stacked tile multiplies only its valid batches' columns (the
                        // valid slots come first): N = count << ln, a multiple of 32
                        const int n = slot_cols[s];
                        id_pos = idesc_f16(n, p.in_fp16, false);
                        id_neg = idesc_f16(n, p.in_fp16, true);
                    }
                    const uint32_t st = smem_u32(smem + s * L::kStage);
#pragma unroll
                    for (int kk = 0; kk < kTcBK / 16; kk++) {
#pragma unroll
                        for (int q = 0; q < 12; q++) {
                            const uint64_t ad = smem_desc_sw64(st + pa[q] * L::kAPlane + kk * 32);
                            const uint64_t bd = smem_desc_sw64(st + 4 * L::kAPlane + pb[q] * L::kBPlane + kk * 32);
                            const uint32_t accum = (kb == 0 && kk == 0 && (q == 0 || q == 6)) ? 0u : 1u;
                            mma_f16(dcol + (acc[q] ? BN : 0), ad, bd, neg[q] ? id_neg : id_pos, accum);
                        }
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                mma_commit(smem_u32(&acc_full[b]));  // also after an abort: flushes issued MMAs
                last_b = b;
                last_par = (uint32_t)((it >> 1) & 1);
            }
            // after an abort, MMAs may still be running: drain them before TMEM is freed
            if (*abort_flag && last_b >= 0) mbar_drain(smem_u32(&acc_full[last_b]), last_par, kLimit);
        }
    } else {
        // epilogue warps 2..9: TMEM lane quarter = warp % 4 = tile rows 32*(warp%4)..; warps
        // 2-5 store columns [0, BN/2) of the tile, warps 6-9 columns [BN/2, BN)
        const int quarter = warp & 3;
        const int c_begin = ((warp - 2) >> 2) * (BN / 2), c_end = c_begin + BN / 2;
        const int row = 32 * quarter + lane;
        const long long M = 1LL << p.lm, N = 1LL << p.ln;
        // scatter(n0 + c0 + j) = scatter(n0 + c0) + scatter(j) for j < 16 (disjoint bits)
        const int lo_bits = min(p.ln, 4);
        long long lo[16];
#pragma unroll
        for (int j = 0; j < 16; j++) lo[j] = scatter_bits(j, p.pos_n, lo_bits);
        int it = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
            const int b = it & 1;
            // the tile's coordinates and output bases first: their loads and bit scatters
            // overlap the wait for the accumulator
            TcTile tt;
            const int *sb = nullptr;  // stacked: this tile's batch indices
            int nonb = 0;
            if (stk) {
                const TcStackTile ts = tc_stack_tile(t, tiles_m, n_stacks, p.ga.nnb);
                tt.tn_i = 0;
                tt.tm_i = ts.tm_i;
                tt.v = ts.v;
                tt.bat = 0;
                sb = p.stack + 2 + (long long)ts.stack * (S + 1);  // the stack's batch indices
                nonb = ts.nonb;
            } else {
                tt = tc_tile(t, tiles_m, tiles_n, p.lbat, p.group_m);
            }
            const int tn_i = tt.tn_i, tm_i = tt.tm_i, bat = tt.bat;
            long long vrow = tt.v;  // this row's version
            long long m;
            if (p.fold == 1) {
                vrow = (long long)tm_i * vm + (row >> p.lm);
                m = row & (M - 1);
            } else {
                m = (long long)tm_i * kTcBM + row;
            }
            const bool row_ok = m < M && vrow < p.nver;
            const long long mbase = row_ok ? scatter_bits(m, p.pos_m, p.lm) : 0;
            long long cbase = scatter_bits(bat, p.pos_bat, p.lbat) + mbase;
            // stacked: this warp's columns cover the stack's batches j0 and (if BN / 2 > N)
            // j0 + 1; their indices (-1: empty) and output bases
            const int j0 = c_begin >> p.ln;
            int be0 = -1, be1 = -1;
            long long cb0 = 0, cb1 = 0;
            if (stk) {
                be0 = j0 < S ? sb[j0] : -1;
                be1 = (j0 + 1 < S && ((j0 + 1) << p.ln) < c_end) ? sb[j0 + 1] : -1;
                if (be0 >= 0) cb0 = scatter_bits(tc_compose_bat(p.ga, p.lbat, nonb, be0), p.pos_bat, p.lbat) + mbase;
                if (be1 >= 0) cb1 = scatter_bits(tc_compose_bat(p.ga, p.lbat, nonb, be1), p.pos_bat, p.lbat) + mbase;
            }
            if (!mbar_wait(smem_u32(&acc_full[b]), (uint32_t)((it >> 1) & 1), abort_flag, kLimit)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * 2 * BN);
            for (int c0 = c_begin; c0 < c_end; c0 += 16) {
                float re[16], im[16];
                // stacked: columns [j N, (j + 1) N) belong to the stack's batch j (N >= 32);
                // an empty slot's columns were not computed (warp-uniform skip)
                const bool first = (c0 >> p.ln) == j0;
                const int be = stk ? (first ? be0 : be1) : 0;
                if (be < 0) continue;
                __syncwarp();
                tmem_ld16x2(lane_addr + c0, lane_addr + BN + c0, re, im);
                if (!row_ok) continue;
                if (stk) {
                    const long long cb = first ? cb0 : cb1;
                    const long long nb = c0 & (N - 1);
                    void *Cv = static_cast<char *>(p.C) + 8 * vrow * p.c_plane;
                    const long long hi = cb + scatter_bits(nb >> 4, p.pos_n + 4, p.ln - 4);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const long long off = hi + lo[j];
                        const float2 x = make_float2(re[j] * p.out_scale, im[j] * p.out_scale);
                        if (p.out_fmt == OUT_C64) static_cast<float2 *>(Cv)[off] = x;
                        else store_split(Cv, p.c_plane, off, x, p.out_fmt == OUT_SPLIT_FP16);
                    }
                    continue;
                }
                if (p.fold == 2) {
                    // columns: version (c0 + j) / N of this tile, n = (c0 + j) % N
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        const long long col = c0 + j;
                        const long long v = (long long)tn_i * vn + (col >> p.ln), n = col & (N - 1);
                        if (v < p.nver) {
                            void *Cv = static_cast<char *>(p.C) + 8 * v * p.c_plane;
                            const long long off = cbase + scatter_bits(n, p.pos_n, p.ln);
                            const float2 x = make_float2(re[j] * p.out_scale, im[j] * p.out_scale);
                            if (p.out_fmt == OUT_C64) static_cast<float2 *>(Cv)[off] = x;
                            else store_split(Cv, p.c_plane, off, x, p.out_fmt == OUT_SPLIT_FP16);
                        }
                    }
                    continue;
                }
                void *Cv = static_cast<char *>(p.C) + 8 * vrow * p.c_plane;
                const long long nb = (long long)tn_i * BN + c0;
                if (nb < N) {
                    const long long hi = cbase + (p.ln > 4 ? scatter_bits(nb >> 4, p.pos_n + 4, p.ln - 4) : 0);
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        if (nb + j < N) {
                            const long long off = hi + lo[j];
                            const float2 x = make_float2(re[j] * p.out_scale, im[j] * p.out_scale);
                            if (p.out_fmt == OUT_C64) static_cast<float2 *>(Cv)[off] = x;
                            else store_split(Cv, p.c_plane, off, x, p.out_fmt == OUT_SPLIT_FP16);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
        }
    }
    __syncwarp();
    if (*abort_flag && threadIdx.x == 0) {
        atomicExch(p.err, 1);
        // let copies already issued land before the shared memory is released
        for (long long k = 0; k < issued && k < STAGES; k++) {
            const long long slot = issued - 1 - k;
            mbar_drain(smem_u32(&full[slot % STAGES]), (uint32_t)((slot / STAGES) & 1), kLimit);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

}  // namespace tnk
