/*
 * tn.h — C-ABI of the GB300 sliced-contraction sampler (libtn.so).
 *
 * Method: arXiv:2112.15083, "Classical Sampling of Random Quantum Circuits with
 * Bounded Fidelity".  Batches of 2^|A| amplitudes of a random circuit are computed by
 * contracting its tensor network once per slice (an assignment of the sliced legs)
 * and summing over a chosen set of slices only (Sec. I.C); the slices are chosen by
 * their norms R[i] = ||psi_i||^2 (Sec. I.A-B, App. B Alg. 1-2); bitstrings are drawn
 * from the batches by modified frugal rejection sampling (Sec. II.A).
 *
 * Conventions shared by every entry point:
 *  - Return codes: TN_OK (0) or a negative TN_E* code.  tn_strerror() names a code;
 *    tn_last_error() gives a detail message for the calling thread's last failure.
 *  - Qubit q of a bitstring is bit q of a uint64 (so at most 64 qubits).
 *  - Wire segments ("vertices", the tensor legs of App. B): single-qubit gates are
 *    merged into the preceding two-qubit gate on their wire (leading ones into the
 *    |0> input), so segment (q, s) is the wire of qubit q just before its (s+1)-th
 *    two-qubit gate, and s = (two-qubit gates on q) is the circuit output of q.
 *    Only internal segments (1 <= s < two-qubit gates on q) can be sliced.
 *  - Open qubits A (the batch, N_A = 2^|A|) are given in an order: bit r of the
 *    in-batch index i is qubit open[r].  Closed qubits B are the others in ascending
 *    order: bit c of a closed pattern j is the c-th closed qubit.
 *  - A slice is a uint64 whose bit e is the value of the e-th sliced edge of the plan.
 *  - Complex numbers are interleaved (re, im) pairs of doubles.
 *  - The caller owns every array it passes; the plan copies what it keeps.  The plan
 *    owns its device memory (see tn_plan_opts.alloc) and enqueues work on
 *    tn_plan_opts.stream; calls return after that work has finished.
 *  - Not thread-safe per plan: one call at a time per plan handle.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TN_OK 0
#define TN_EINVAL (-1)       /* bad argument, circuit, order or slice set */
#define TN_ENOMEM (-2)       /* host or device allocation failed, or the HBM budget is exceeded */
#define TN_ETIMEOUT (-3)     /* a bounded device-side wait gave up */
#define TN_EDEVICE (-4)      /* CUDA error (no device, launch failure, ...) */
#define TN_EUNSUPPORTED (-5) /* valid request outside what libtn implements */

/* Precision of the pairwise contractions: complex64, or each operand split into a hi and a
   lo part of a narrow type whose products are summed in FP32 (hi*hi + hi*lo + lo*hi). */
#define TN_PREC_C64 0    /* complex64 operands, FP32 FFMA accumulation */
#define TN_PREC_BF16X2 1 /* hi+lo bf16 split operands on tcgen05, FP32 accumulation */
#define TN_PREC_FP16X2 2 /* hi+lo fp16 split operands (scaled) on tcgen05, FP32 accumulation */

/* Flags for buffers passed to tn_contract / tn_sample. */
#define TN_DEVICE_BUFFERS 1 /* closed_bits / amps / bitstrings are device pointers */

typedef struct tn_circuit_s *tn_circuit_h;
typedef struct tn_plan_s *tn_plan_h;

typedef struct {
    int32_t qubit;
    int32_t segment;
} tn_edge;

/* Device memory provider.  alloc returns NULL on failure; both run on the host
 * thread that made the call.  A NULL alloc means cudaMallocAsync/cudaFreeAsync on
 * the plan's stream. */
typedef void *(*tn_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*tn_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct {
    int32_t precision;       /* TN_PREC_* */
    int32_t log2_batches;    /* batches contracted together: T = 2^log2_batches (0..16) */
    uint64_t order_seed;     /* seed of the randomised greedy contraction order */
    int32_t order_trials;    /* greedy trials (best estimated time wins); <= 0: 64 */
    int32_t n_auto_sliced;   /* when sliced == NULL: how many edges the planner slices */
    int32_t max_log2_tensor; /* when sliced == NULL and > 0: instead, slice edges until no
                                tensor of one slice exceeds 2^max_log2_tensor elements
                                (for circuits run a few slices at a time); 0: off */
    double hbm_budget_bytes; /* device working-set limit per call; <= 0: 64 GiB */
    double max_norm_flops;   /* tn_partial_norms refuses norm networks above this many
                                algorithmic FLOPs (TN_EUNSUPPORTED); <= 0: 2e15 */
    int32_t autotune;        /* 1 (default): the first execution of each step shape times
                                every applicable kernel variant (FFMA tile shape, row or
                                staged kernel, tensor-core tile width) and keeps the
                                fastest; the choice is cached per shape for the process.
                                0: fixed shape rules.  k >= 2: step i runs variant
                                (i + k - 2) mod (its variant count), so that tests can run
                                every variant.  All variants accumulate each output over k
                                in the same order. */
    int32_t fuse_root_sum;   /* 1: when the root step runs the row kernel, run it fused
                                with the FP64 slice sum (Sec. I.C step 1) in one launch
                                whose output is bit-identical to the two launches, without
                                writing the root's per-slice values to memory.  0
                                (default): separate launches. */
    int32_t job_groups;      /* batch groups per sampling job that the order search
                                optimises for: a batch-independent step runs once per
                                job, the others once per group; <= 1 (default): one */
    int32_t anneal_iters;    /* order search: simulated-annealing moves (tree rotations,
                                Metropolis on the log of the estimated time) applied to
                                the winning tree, kept only if cheaper; 0 (default): none */
    int32_t parallel_search; /* 1: the greedy trials draw from per-trial generators and run
                                on host threads (faster planning; other trees than the
                                default, equally seeded and reproducible); 0 (default):
                                one sequential generator */
    void *stream;            /* cudaStream_t; NULL = legacy default stream */
    tn_alloc_fn alloc;       /* optional device allocator */
    tn_free_fn free;
    void *alloc_ctx;
} tn_plan_opts;

/* Fill opts with the defaults above (C64, T = 256, seed 0, 64 trials, 64 GiB). */
void tn_plan_opts_default(tn_plan_opts *opts);

/* Parse a serialized circuit: b"RQC1", uint32 n_qubits, uint32 n_gates, then per gate
 * uint32 arity (1|2), uint32 q0, uint32 q1 (0xFFFFFFFF if arity 1) and (2^arity)^2
 * complex128 matrix entries, row-major; a two-qubit basis index is 2*bit(q0)+bit(q1).
 * (The circuit C of Sec. I.A; gates are the tuples (l, A, q) of App. B.)
 * Errors: TN_EINVAL on a malformed buffer or more than 64 qubits. */
int tn_circuit_load(const void *buf, size_t len, tn_circuit_h *out);
void tn_circuit_destroy(tn_circuit_h c);

/*
 * Build a contraction plan: the tensor network of C with the open qubits' output legs
 * left open and the closed ones bound to a batch-indexed selector, a contraction tree
 * (Sec. I, "contraction tree"), the sliced legs I (Sec. I, "sliced variables") and a
 * compiled list of pairwise contractions, each a batched complex GEMM whose output is
 * written in the layout its consumer reads.
 *
 *  order        NULL, or 2*(n_leaves-1) int32 giving the contraction tree as SSA pairs:
 *               leaves are the merged two-qubit gates in circuit order, then one leaf
 *               per qubit without two-qubit gates; each pair creates the next id.
 *  sliced       NULL (the planner picks opts->n_auto_sliced edges) or n_sliced internal
 *               wire segments, n_sliced <= 62.
 *  open_qubits  n_open distinct qubits (n_open <= 16); the batch size is 2^n_open.
 * Errors: TN_EINVAL (bad order / segment / qubit), TN_ENOMEM, TN_EDEVICE.
 */
int tn_plan(tn_circuit_h c, const int32_t *order, int32_t n_order, const tn_edge *sliced,
            int32_t n_sliced, const int32_t *open_qubits, int32_t n_open,
            const tn_plan_opts *opts, tn_plan_h *out);
void tn_plan_destroy(tn_plan_h p);

typedef struct {
    int32_t n_qubits, n_open, n_closed, log2_batches;
    int32_t n_leaves, n_steps, n_sliced;
    int32_t log2_max_tensor;     /* largest per-slice intermediate (elements, log2) */
    double flops_per_slice;      /* 8 * sum over steps of prod(dims), one slice, one group */
    double flops_all_slices;     /* same, summed with reuse over all 2^n_sliced slices */
} tn_plan_info;

int tn_plan_get_info(tn_plan_h p, tn_plan_info *info);
/*
 * Host-only planning (no device work), for inspection and tests: runs the same planner
 * as tn_plan and fills info; if steps != NULL, writes up to cap_steps rows of seven
 * int32 per step (batch bits, m bits, n bits, k bits, then log2 of the versions of C, A
 * and B over the full slice set);
 * if sliced_out != NULL, writes up to cap_sliced sliced edges in slice-bit order.
 */
int tn_plan_host(tn_circuit_h c, const int32_t *order, int32_t n_order, const tn_edge *sliced,
                 int32_t n_sliced, const int32_t *open_qubits, int32_t n_open,
                 const tn_plan_opts *opts, tn_plan_info *info, int32_t *steps, int32_t cap_steps,
                 tn_edge *sliced_out, int32_t cap_sliced);

/*
 * App. B Alg. 2 SlicedVertexSelect(C, I, k) on the host: greedy choice of S in I, each
 * step taking the candidate u outside S and L'_C(S) that minimises |L'_C(S + {u})|
 * (ties: first in I), then dropping from S the vertices u depends on.  Vertices are wire
 * segments; s_index receives positions into I of S in (qubit, segment) order.
 */
int tn_sliced_vertex_select(tn_circuit_h c, const tn_edge *I, int32_t n_I, int32_t k,
                            int32_t *s_index, int32_t *k_out);

/* The plan's sliced edges I in slice-bit order (cap entries at most). */
int tn_plan_sliced_edges(tn_plan_h p, tn_edge *out, int32_t cap, int32_t *n_out);

/*
 * Partial-slice norms (Sec. I.A, App. B Alg. 1 steps 1-3): S = SlicedVertexSelect(C, I,
 * k0) with k0 = ceil(3 - log2 f) (Alg. 2), C1 = union of the lightcones of S, and
 * R[i] = <0|C1* delta_{S=i} C1|0> = ||psi_i||^2 for i in {0,1}^k, computed on the GPU
 * by contracting the network C1 (x) C1* with the S legs identified (Fig. 1) in the plan's
 * contraction precision (complex64, or the split tensor-core path), summed in FP64.
 *  s_index  out, k entries: positions of S within the plan's sliced edges (ascending);
 *           bit t of i is S[t].
 *  R        out, host, cap_R >= 2^k doubles.
 * Errors: TN_EINVAL (f outside (0,1], cap too small), TN_EUNSUPPORTED (the norm network's
 * contraction would exceed tn_plan_opts.max_norm_flops; checked before any device work),
 * TN_EDEVICE.
 */
int tn_partial_norms(tn_plan_h p, double f, int32_t *s_index, int32_t *k, double *R,
                     int64_t cap_R);

/*
 * Slice cut (Alg. 1 steps 4-5) on the GPU: sort R descending (ties: index ascending),
 * sum in that order in FP64, keep the minimal prefix whose sum reaches f (all of it if
 * rounding keeps the total below f).  R: host array of 2^k doubles.  X: out, host,
 * the kept indices in sorted order (cap 2^k); F: the kept sum.  k <= 12 (one block sorts
 * the 2^k norms in shared memory); larger k returns TN_EINVAL.  The device scratch is
 * allocated and freed on the stream inside the call, which synchronises the stream.
 */
int tn_slice_cut(const double *R, int32_t k, double f, void *stream, int32_t *X,
                 int32_t *n_x, double *F);

/*
 * tn_slice_cut without any device allocation (the paper has no counterpart; this is a
 * deployment variant).  For callers that cannot allocate device memory from their call
 * path: processes whose device memory is owned up front by another allocator, and code
 * that must not enter the CUDA allocator (which can wait on other device work and can
 * fail under fragmentation).  Same arguments, results and limit (k <= 12, TN_EINVAL
 * above) as tn_slice_cut.  The device scratch is a static array in libtn of 48 KiB +
 * 256 B (2^12 doubles, 2^12 int32, the count and the sum) that every GPU loading the
 * library holds until the process exits.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and caches it
 * per device ordinal; the cache is not valid across cudaDeviceReset.  The call
 * synchronises the stream, so it cannot be made while the stream is being captured.
 * All calls share the one array per device: calls whose work overlaps on the GPU race
 * with each other.
 */
int tn_slice_cut_noalloc(const double *R, int32_t k, double f, void *stream, int32_t *X,
                         int32_t *n_x, double *F);

/*
 * Slice selection for fidelity f (Alg. 1): tn_partial_norms + tn_slice_cut, then the
 * slice set X x {0,1}^{|I|-k} (Sec. I.C step 1) written to slices (cap entries).  When
 * f >= 1 every slice is kept and F = 1.  n_slices receives the set size even if cap is
 * too small (then TN_EINVAL).
 */
int tn_select(tn_plan_h p, double f, uint64_t *slices, int64_t cap, int64_t *n_slices,
              double *F);

/*
 * Host-only estimate for a slice set (no device work): device_bytes = arena + leaves +
 * per-group buffers (+ 64 MiB slack); flops_first / flops_next = algorithmic FLOPs of the
 * first batch group and of each later group (which reuses the batch-free stem).
 */
int tn_plan_estimate(tn_plan_h p, const uint64_t *slices, int64_t n_slices, int64_t *device_bytes,
                     double *flops_first, double *flops_next);

/*
 * Amplitudes of n_batches batches summed over a slice set (Sec. I.C step 1; no
 * normalisation): amps[t*2^n_open + i] = sum over slices s of <i, closed_bits[t]|C_s|0>,
 * C_s the network with the sliced legs fixed by s.  Slices are summed in FP64 in the
 * given order.  Slices must be distinct; closed_bits holds one pattern per batch.
 *  flags & TN_DEVICE_BUFFERS: closed_bits and amps are device pointers, else host.
 * Errors: TN_EINVAL (duplicate or out-of-range slice), TN_ENOMEM (budget), TN_EDEVICE.
 */
int tn_contract(tn_plan_h p, const uint64_t *slices, int64_t n_slices, const uint64_t *closed_bits,
                int64_t n_batches, double *amps, int32_t flags);

/*
 * Verification (linear XEB, Eq. 1): the
 * amplitude a(s) of each of N bitstrings summed over a slice set (unnormalised, as
 * tn_contract computes it) and their linear XEB, xeb = 2^n / N * sum_s |a(s)|^2 - 1.
 * A string's closed qubits select its batch and its open qubits its entry; a plan with no
 * open qubits computes one amplitude per string.  Groups after the first reuse the
 * batch-independent contractions.  The sum of |a|^2 = re*re + im*im (no fused
 * multiply-add) runs in FP64 on the device in a fixed order.
 *  bitstrings  N host values (bit q = qubit q, below the circuit's qubit count).
 *  amps        NULL, or N host complex128 values (interleaved) receiving a(s).
 * Errors: TN_EINVAL (bad slice or bitstring), TN_ENOMEM (budget), TN_EDEVICE.
 */
int tn_xeb(tn_plan_h p, const uint64_t *slices, int64_t n_slices, const uint64_t *bitstrings, int64_t N,
           double *xeb, double *amps);

/*
 * XEB spoofing (Sec. III, "Spoofing Linear XEB"): the amplitudes of one batch (the closed
 * qubits fixed to closed_pattern, all 2^n_open open patterns) summed over a slice set,
 * then the N strings of largest p = re*re + im*im (FP64, no fused multiply-add; equal
 * values: the smaller in-batch index first), selected exactly on the device (radix select
 * of the FP64 bit patterns).  The recipe takes n_open = ceil(log2(10 N)) and the slice set
 * of tn_select at the target fidelity; a plan with log2_batches = 0 computes that batch
 * alone.
 *  bitstrings  out, N entries in ascending in-batch index order (bit q = qubit q).
 *  probs       NULL, or out: p of each selected string (unnormalised).
 * Errors: TN_EINVAL (N outside [1, 2^n_open], n_open > 30, bad pattern or slices).
 */
int tn_spoof(tn_plan_h p, const uint64_t *slices, int64_t n_slices, uint64_t closed_pattern, int64_t N,
             uint64_t *bitstrings, double *probs);

typedef struct {
    double F;           /* retained fidelity sum_{i in X} R[i] (1 when f >= 1) */
    double eps_hat;     /* Sec. II.C: eps_J / |J| over the computed batches */
    int64_t steps;      /* batches computed (|J|) */
    int64_t accepted;   /* accepted batches (>= N unless max steps reached) */
    int64_t n_slices;   /* size of the contracted slice set */
    double flops;       /* algorithmic FLOPs of the contractions (8 * complex MACs) */
} tn_sample_stats;

/*
 * Sampling with fidelity (Sec. II.A): select slices for f_target (Alg. 1), then for
 * t = 0, 1, ... draw j_t uniformly, contract the batch j_t over the slices, set
 * p_{i,j} = |a_{i,j}|^2 / F, accept with probability min(1, p_j N_B / alpha) and pick i
 * with probability p_{i,j}/p_j.  Batches are processed 2^log2_batches at a time until N
 * are accepted (at most ceil(8 alpha N) + 4096 batches).  When the selected slice set does
 * not fit the plan's HBM budget in one execution, the call runs a sampling job instead
 * (tn_job_create with automatic chunks, every chunk, tn_job_finish).  Random numbers: Philox4x32-10
 * with key = seed and counter = (t, stream): stream 0 gives j (low |B| bits of words
 * 0-1) and u (words 2-3), stream 1 gives v; a 64-bit word w maps to (w >> 11) 2^-53.
 * Accept iff u*alpha < p_j*N_B.  Requires n_open = 6.
 *  bitstrings  out, N entries, the accepted strings in t order.
 *  alpha       > 1 (paper: 2).
 */
int tn_sample(tn_plan_h p, double f_target, int64_t N, uint64_t seed, double alpha,
              uint64_t *bitstrings, int32_t flags, tn_sample_stats *stats);

/*
 * Sampling job over a slice set larger than one execution's memory (Sec. I.C step 1 with
 * Sec. II.A).  The retained slices X x {0,1}^{|I|-k} of tn_select are split into chunks
 * of chunk_slices slices that differ only in the same free legs (those that add the least
 * work when they vary inside a chunk: the steps that do not depend on them run once per
 * chunk);
 * the job's batches t = 0 .. groups * T - 1 (T = 2^log2_batches) are drawn once (Philox,
 * as in tn_sample).  tn_job_run contracts chunks for every batch group: per chunk the
 * batch-independent intermediates are computed once and reused by all groups, and each
 * group's sum over the chunk's slices is added in FP64 to that group's amplitudes, chunk
 * after chunk in chunk order.  tn_job_finish then runs the accept / pick step of
 * tn_sample on all batches (p = |a|^2 / F) and returns the first N accepted strings in t
 * order.  groups = ceil((1.1 alpha N + 8 sqrt(alpha N) + 64) / T) batches are drawn, so
 * that N accepted strings are all but certain; TN_EINVAL reports a shortfall.
 * The job owns device buffers of groups * T * (64 * 16 + 8) bytes (from the plan's
 * allocator) until tn_job_destroy.  Requires n_open = 6.
 */
typedef struct tn_job_s *tn_job_h;

typedef struct {
    int64_t n_slices;      /* retained slices */
    double F;              /* their fidelity (Alg. 1) */
    int64_t chunk_slices;  /* slices per chunk */
    int64_t n_chunks;
    int64_t groups;        /* batch groups of T batches */
    int64_t T;             /* batches per group */
    int64_t chunks_done;   /* chunks contracted so far */
    double flops_done;     /* algorithmic FLOPs of the chunks contracted so far */
    double flops_chunk;    /* algorithmic FLOPs of one chunk over all groups (stem once) */
} tn_job_info;

/*
 * Create a job for N samples at fidelity f_target.  The chunk is the largest power of two
 * of slices whose working set (tn_plan_estimate) plus the job's buffers fits 95% of the
 * plan's HBM budget; max_chunk_slices > 0 caps it further.
 * Errors: TN_EINVAL (arguments, n_open != 6), TN_ENOMEM (not even one slice fits).
 */
int tn_job_create(tn_plan_h p, double f_target, int64_t N, uint64_t seed, double alpha,
                  int64_t max_chunk_slices, tn_job_h *out, tn_job_info *info);

/* Contract chunks first .. first + count - 1 for every group and add them to the job's
 * amplitudes; synchronises.  Each chunk may run once (TN_EINVAL otherwise). */
int tn_job_run(tn_job_h j, int64_t first, int64_t count);

int tn_job_get_info(tn_job_h j, tn_job_info *info);

/* The accumulated amplitudes of group g (T * 64 complex128, batch-major), unnormalised,
 * into a host array; synchronises. */
int tn_job_amplitudes(tn_job_h j, int64_t g, double *amps);

/*
 * Accept / pick over every batch of the job and the first N accepted strings in t order
 * (host array; stats as tn_sample).  Unless flags & TN_JOB_PARTIAL, every chunk must have
 * run (TN_EINVAL otherwise); with it, the sums over the chunks run so far are sampled
 * (not the target distribution: for timing only) and fewer than N accepted strings is not
 * an error (stats->accepted says how many were written).
 */
#define TN_JOB_PARTIAL 2
int tn_job_finish(tn_job_h j, uint64_t *bitstrings, int32_t flags, tn_sample_stats *stats);

void tn_job_destroy(tn_job_h j);

/*
 * One sampling step over one batch group (Sec. II.A for t = t0 .. t0 + T - 1, T =
 * 2^log2_batches): draw j_t (Philox, as in tn_sample), contract the T batches over the
 * given slice set, set p = |a|^2 / F, run the accept / pick step and write accept[t] (0/1)
 * and bits[t] (the bitstring (i_t, j_t)).  reuse_stem != 0 skips the contractions that do
 * not depend on the batch (kept from the previous step on the same slice set).
 * flags & TN_DEVICE_BUFFERS: accept / bits are device arrays and the call returns without
 * synchronising the stream; otherwise they are host arrays and the call synchronises.
 */
int tn_sample_step(tn_plan_h p, const uint64_t *slices, int64_t n_slices, double F, uint64_t seed,
                   uint64_t t0, double alpha, int32_t reuse_stem, uint8_t *accept, uint64_t *bits,
                   int32_t flags);

/*
 * Test hook for failure detection (the paper has no counterpart).  With cycles > 0, every
 * tensor-core launch of the plan's later executions first makes its MMA warp wait on a
 * shared-memory barrier that nothing arrives on, giving up after about `cycles` SM clock
 * cycles.  The launch then takes its bounded-wait exit: the CTA records the error word,
 * waits (bounded) for the tile copies it already issued, frees its tensor memory and
 * returns, and the call that synchronises reports TN_ETIMEOUT with the outputs undefined.
 * cycles = 0 restores normal operation; the plan stays usable.  cycles <= 4e9.
 */
int tn_plan_test_stall(tn_plan_h p, int64_t cycles);

/* Tracing: when on, every execution records CUDA events around each contraction step
 * and around the FP64 slice sum on the plan's stream.  tn_trace_read synchronises and
 * reports, per step, the launches, the summed device time, and the algorithmic FLOPs
 * (8 per complex multiply-add) and bytes (operands read + result written, complex64) of
 * one launch; entry n_steps (the last) is the slice sum (FLOPs = FP64 additions). */
typedef struct {
    int32_t step;
    int32_t launches;
    double ms;
    double flops_per_launch;
    double bytes_per_launch;
    int32_t nbat, nm, nn, nk;
    int64_t nver;
    int32_t kernel; /* 0: row kernel, 1: staged small products, 2: FP64 slice sum,
                       3: the root step fused with the FP64 slice sum (the root step's
                       own entry then counts no launches), 4: row kernel with rows
                       staged through shared memory, 5: long-K kernel (at most 8 x 32
                       outputs per batch, K >= 1024), 9128 / 9064 / 9032:
                       tensor-core kernel with 128- / 64- / 32-column tiles,
                       19128 / 19064: stacked tensor-core tiles of 128 / 64 columns (the
                       batches of a group that read the same stored block of an in-place
                       operand, 2 to 4 side by side; each launch is preceded by one
                       launch that builds the group's stack list),
                       TM*1000+TN: FFMA tile kernel */
    int32_t gathers;  /* batch-gather launches that precede each launch of the step (0 or
                         1; 0 when the kernel reads its gathered operands in place) */
    int32_t in_place; /* 1: the step has gathered operands and its kernel reads them in
                         place (row and long-K kernels through the gather's tables,
                         tensor-core kernels through a tensor map over the stored form) */
} tn_step_trace;
int tn_trace_enable(tn_plan_h p, int32_t on);
int tn_trace_read(tn_plan_h p, tn_step_trace *out, int32_t cap, int32_t *n_out);

/*
 * The sampler step alone (Sec. II.A steps 2-3) on given probabilities: p is a device
 * array of T*64 doubles (p[t*64 + i] = p_{i,j_t}, batch index t0 + t); writes accept[t]
 * (0/1) and pick[t] (device arrays).  The batch total and prefix sums use a 32-lane
 * Kogge-Stone scan of pair sums (offsets 1,2,4,8,16); p_j is the last lane's total; the
 * pick is the smallest i whose prefix exceeds v*p_j, else the last i with p_i > 0.
 */
int tn_rejection_sample(const double *p, int64_t T, int32_t b_bits, double alpha, uint64_t seed,
                        uint64_t t0, uint8_t *accept, int32_t *pick, void *stream);

/* Batch draws j_t = low b_bits of Philox(seed, t0 + t, stream 0) words 0-1 (device out). */
int tn_draw_batches(uint64_t seed, uint64_t t0, int64_t T, int32_t b_bits, uint64_t *j,
                    void *stream);

/* Synchronise the plan's stream and report a deferred device error (a bounded device wait
 * that gave up during asynchronous tn_sample_step calls): TN_OK or TN_ETIMEOUT. */
int tn_plan_sync(tn_plan_h p);

/* ------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop above this C-ABI.  Requests (circuit, open
 * qubits, precision, target fidelity f, N samples, seed, alpha) are planned on planner
 * threads (tn_plan, tn_select, tn_plan_estimate), admitted while the sum of admitted
 * device-memory estimates stays within hbm_budget_bytes and at most max_active run, and
 * advanced one batch group (tn_sample_step) at a time on their own CUDA streams, so the
 * groups of different requests overlap on the device.  A request's samples depend only on
 * its own inputs (deterministic plan, counter-based draws, fixed-order sums), so they are
 * the same alone and in any mix.  Requests whose estimated GPU time (FLOPs of all batch
 * groups / assumed_flops) exceeds max_request_seconds are rejected (TN_REQ_REJECTED).
 * (The paper describes no serving layer; this is a deployment component.)
 * ---------------------------------------------------------------------------------- */
typedef struct tn_server_s *tn_server_h;

typedef struct {
    double hbm_budget_bytes;    /* admission budget (default 150e9) */
    int32_t max_active;         /* requests running at once (default 8) */
    int32_t planner_threads;    /* default 2 */
    int32_t log2_batches;       /* smallest batch group of a request (default 8) */
    int32_t max_log2_batches;   /* largest: a request of N samples gets the smallest group
                                   of at least 1.1 alpha N batches within these bounds, since
                                   the batches of a group share their batch-independent
                                   intermediates (default 14) */
    int32_t order_trials;       /* order-search trials per plan (default 64); served plans
                                   use the fixed kernel shape rules (no autotuning) */
    double max_request_seconds; /* estimated-time limit per request (default 600); it also caps
                                   the norm network of the slice selection */
    double assumed_flops;       /* rate of split-precision plans for that estimate (3e14) */
    double assumed_flops_c64;   /* rate of complex64 plans (default 3e13 FLOP/s) */
    int32_t device;             /* CUDA device (default 0) */
} tn_server_opts;

#define TN_REQ_QUEUED 0
#define TN_REQ_PLANNING 1
#define TN_REQ_PLANNED 2
#define TN_REQ_ACTIVE 3
#define TN_REQ_DONE 4
#define TN_REQ_FAILED 5
#define TN_REQ_REJECTED 6

typedef struct {
    int32_t status;             /* TN_REQ_* */
    int32_t error;              /* TN_OK or the failing call's code */
    double F;                   /* retained fidelity of the slice set */
    int64_t steps, accepted;    /* batches computed and accepted */
    int64_t n_slices;
    int64_t est_bytes;          /* admission estimate */
    double flops;               /* algorithmic FLOPs spent */
    double t_submit, t_admit, t_done; /* seconds since the server was created */
} tn_request_info;

typedef struct {
    int64_t submitted, queued, planning, planned, active, done, failed, rejected;
    double bytes_in_use;        /* sum of the admitted requests' estimates */
    double time_s;              /* seconds since the server was created */
} tn_server_stats;

void tn_server_opts_default(tn_server_opts *opts);
int tn_server_create(const tn_server_opts *opts, tn_server_h *out);
/* Non-blocking; circuit is copied.  n_sliced: legs the planner slices (tn_plan_opts.n_auto_sliced). */
int tn_server_submit(tn_server_h s, const void *circuit, size_t len, const int32_t *open_qubits,
                     int32_t n_open, int32_t precision, int32_t n_sliced, double f, int64_t N,
                     uint64_t seed, double alpha, int64_t *id);
int tn_server_query(tn_server_h s, int64_t id, tn_request_info *info);
/* Blocks until the request ends (timeout_s <= 0: no limit; else TN_ETIMEOUT); copies up to
 * cap bitstrings (the first N accepted, in t order) when it succeeded. */
int tn_server_wait(tn_server_h s, int64_t id, double timeout_s, uint64_t *bitstrings, int64_t cap,
                   tn_request_info *info);
int tn_server_get_stats(tn_server_h s, tn_server_stats *stats);
/* Cancels queued requests, finishes active ones, joins the threads. */
void tn_server_destroy(tn_server_h s);

const char *tn_strerror(int code);
const char *tn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
