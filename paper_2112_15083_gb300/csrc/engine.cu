// libtn executor and C-ABI (see include/tn.h).
//
// A plan holds the compiled amplitude network (leaves on the device, a step list) and
// executes a slice set as follows: every tree node x gets one version per distinct
// projection of the slice set on the sliced legs below x (so intermediates shared by
// several slices are computed once); each step is one launch over all versions; the
// root versions are summed in FP64 in slice order (Sec. I.C).  Leaves holding closed
// output legs are re-materialised per batch group with the group's closed patterns.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <type_traits>
#include <unordered_map>

#include <cudaTypedefs.h>

#include "arena.h"
#include "gather_tables.h"
#include "kernels.cuh"
#include "tc.cuh"
#include "tn_internal.h"

namespace {
thread_local std::string g_err;
}
void tn_set_error(const std::string &m) { g_err = m; }

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) {                                                                \
            tn_set_error(std::string("CUDA error: ") + cudaGetErrorString(e_) + " in " #x);     \
            return TN_EDEVICE;                                                                  \
        }                                                                                       \
    } while (0)

#define RC(x)                       \
    do {                            \
        int r_ = (x);               \
        if (r_ != TN_OK) return r_; \
    } while (0)

namespace {

struct DevMem {
    tn_alloc_fn alloc = nullptr;
    tn_free_fn free = nullptr;
    void *ctx = nullptr;
    cudaStream_t stream = nullptr;
    void *get(size_t bytes) {
        bytes = std::max<size_t>(bytes, 256);
        void *p = nullptr;
        if (alloc) p = alloc(bytes, stream, ctx);
        else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) p = nullptr;
        return p;
    }
    void put(void *p, size_t bytes) {
        if (!p) return;
        bytes = std::max<size_t>(bytes, 256);
        if (free) free(p, bytes, stream, ctx);
        else cudaFreeAsync(p, stream);
    }
};

struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

int ensure(DevMem &mem, DBuf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return TN_OK;
    mem.put(b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = std::max<size_t>(bytes, 256);
    b.p = mem.get(want);
    if (!b.p) {
        tn_set_error("device allocation of " + std::to_string(want) + " bytes failed");
        return TN_ENOMEM;
    }
    b.bytes = want;
    return TN_OK;
}

void release(DevMem &mem, DBuf &b) {
    mem.put(b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
}

// A buffer released when the scope ends, on error returns too.
struct ScopedBuf {
    DevMem &mem;
    DBuf b;
    explicit ScopedBuf(DevMem &m) : mem(m) {}
    ~ScopedBuf() { release(mem, b); }
    ScopedBuf(const ScopedBuf &) = delete;
    ScopedBuf &operator=(const ScopedBuf &) = delete;
};

// Versions and memory layout of one execution of a compiled network on a slice set.
struct CallPlan {
    std::vector<uint64_t> slices;              // key
    std::vector<long long> nver;               // per node
    std::vector<size_t> off;                   // arena byte offset per internal node
    std::vector<size_t> tab_off;               // per step: index of ptrA table in tables
    size_t root_tab = 0;                       // index of the root table
    std::vector<const void *> host_tab;        // pointer tables (device addresses)
    size_t arena_bytes = 0;
    double flops_all = 0, flops_beta = 0;      // per execution (all steps / beta steps)
    long long root_nver = 0;                   // explicit root versions (slice sum outer loop)
    std::vector<size_t> map_off;               // per step: first tensor map (A, B)
    std::vector<CUtensorMap> maps;
    std::vector<size_t> vidx_off;              // per step: offset into the version index table
    std::vector<int> fold;                     // per step: 0, 1 (versions into M), 2 (into N)
    std::vector<std::array<char, 2>> tc_inplace;  // per step and operand: tensor-core map over the
                                                  // stored form of a gathered operand (no copy)
    std::vector<int> vidx;                     // host copy; device copy in CNet::vidx_dev
    std::vector<std::array<size_t, 2>> goff;   // per step: arena offsets of gathered operands
    std::vector<tnk::GatherDesc> gd;           // batch gathers (device copy in CNet::gdescs)
    std::vector<size_t> gd_off;                // per step: first gather descriptor
    std::vector<uint64_t> gtab;                // their lookup tables (device copy in CNet::gtabs)
    bool valid = false;
};

struct CNet {
    Network net;
    Tree tree;
    std::vector<Step> steps;
    uint64_t E = 0;            // explicit-version sliced legs of the compiled variant
    bool compiled = false;
    int prec = TN_PREC_C64;    // precision mode of the tensor-core steps
    int prec_active = -1;      // formats currently materialised (bf16 while calibrating fp16)
    bool calibrated = false;   // fp16 scales measured
    bool calibrating = false;  // this execution records per-node maxima
    DBuf absmax;               // per node: calibration maxima (float bits)
    std::vector<int> fmt;      // per node: storage format (tnk::OutFmt)
    std::vector<float> scale;  // per node: stored value = true value * scale
    std::vector<char> use_tc;  // per step: tcgen05 kernel
    std::vector<int> variant;  // per step: kernel variant (-1: not chosen yet)
    const uint64_t *cur_closed = nullptr;  // batch patterns of the execution being issued
    int autotune = 1;          // 1: time the applicable variants of unseen step shapes;
                               // 0: fixed shape rules; k >= 2: variant (step + k - 2) mod count
    bool fuse_root = false;    // run a row-kernel root step fused with the slice sum
    long long tc_stall = 0;    // tests only: tensor-core launches first wait this many cycles
                               // on a barrier nothing arrives on (see tn_plan_test_stall)
    DBuf err;                  // device error word of the bounded waits
    int *d_err = nullptr;
    // CUDA graphs of one execution (index: stem reuse off / on), valid for the current
    // call plan and the (closed-pattern, output) buffers they were captured with
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    const void *graph_key[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int elem = 8;  // 8: complex64, 16: complex128
    std::vector<DBuf> leaf_src, leaf_dst;
    std::vector<int> leaf_codebits;
    std::vector<std::vector<int>> leaf_sl;  // sliced legs (e) in leg order
    DBuf arena, tables, vidx_dev, gdescs, gtabs;
    DBuf stacks;  // stacked tensor-core tiles: the group's stack list (tnk::tc_stack_build)
    CallPlan cp;
    std::vector<int> parent;
    size_t leaf_bytes = 0;
    // tracing
    bool trace = false;
    std::vector<cudaEvent_t> ev;        // 2 per step
    std::vector<int> ev_pending;        // per step: events recorded and not yet read
    std::vector<int> tr_launches;
    std::vector<double> tr_ms;
    std::vector<int> tr_kernel;
};

}  // namespace

struct tn_plan_s {
    tn_circuit_s circ;
    Merged mg;
    tn_plan_opts opts{};
    DevMem mem;
    std::vector<tn_edge> I;
    std::vector<int> open, closed;
    int log2T = 0;
    CNet amp;
    DBuf d_closed, d_amps, d_j, d_acc, d_pick, d_eps, d_bits, d_R, d_X;
    DBuf d_xidx, d_xamps, d_xsum;  // tn_xeb: in-batch entries, the strings' amplitudes, sums
    DBuf d_skey, d_shist, d_sgt, d_seq, d_sbits, d_sprob;  // tn_spoof: keys, histogram, counts, output
    double budget = 0;
    // norm cache
    double norm_f = -1;
    std::vector<int> norm_S;
    std::vector<double> norm_R;
};

// ---------------------------------------------------------------- leaves

namespace {

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

// Tensor-core eligibility of a step: K >= 16 (TMA row pitch >= 32 B, one MMA K step)
// and both output dimensions >= 64 (the tile is 128 x 128).
bool tc_step(const Step &s) { return tn_tc_shape(s.nm, s.nn, s.nk); }

// Storage format of every node = what its consumer reads; use_tc[i] != 0 marks the
// steps run on the tensor cores (decided from the per-version shapes, or at call time
// with version folding, see prepare_call).
void apply_formats(CNet &cn, const std::vector<char> &use_tc) {
    const int NN = (int)cn.tree.nodes.size();
    cn.fmt.assign(NN, tnk::OUT_C64);
    if (!(cn.calibrated && (int)cn.scale.size() == NN)) cn.scale.assign(NN, 1.0f);
    cn.use_tc.assign(cn.steps.size(), 0);
    if (cn.prec_active < 0) cn.prec_active = cn.prec == TN_PREC_FP16X2 ? TN_PREC_BF16X2 : cn.prec;
    if (cn.elem != 8 || cn.prec_active == TN_PREC_C64) return;
    const int split = cn.prec_active == TN_PREC_FP16X2 ? tnk::OUT_SPLIT_FP16 : tnk::OUT_SPLIT_BF16;
    for (size_t i = 0; i < cn.steps.size(); i++) {
        const Step &s = cn.steps[i];
        if (!use_tc[i]) continue;
        cn.use_tc[i] = 1;
        cn.fmt[s.a] = split;
        cn.fmt[s.b] = split;
    }
    if (split != tnk::OUT_SPLIT_FP16)
        for (auto &x : cn.scale) x = 1.0f;
    else
        for (int x = 0; x < NN; x++)
            if (cn.fmt[x] != tnk::OUT_SPLIT_FP16) cn.scale[x] = 1.0f;
}

void assign_formats(CNet &cn) {
    std::vector<char> u(cn.steps.size(), 0);
    for (size_t i = 0; i < cn.steps.size(); i++) u[i] = tc_step(cn.steps[i]) ? 1 : 0;
    apply_formats(cn, u);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

std::mutex g_encode_mu;

int get_encoder() {
    std::lock_guard<std::mutex> lock(g_encode_mu);
    if (g_encode) return TN_OK;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        !fn) {
        tn_set_error("cuTensorMapEncodeTiled is not available from the driver");
        return TN_EDEVICE;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return TN_OK;
}

// 4-D map of a split operand: [versions][4 * BAT planes][rows][K] of 2-byte elements
// (a version is 8 bytes per element: four planes), tiles of 32 (K) x 128 rows, 64-byte
// swizzle; out-of-range rows/columns read as zero.
// Stacked tensor-core tiles sort a group's batch indices in shared memory (8 bytes each):
// up to 2^14 batches per group.
constexpr int kStackMaxBeta = 14;

int encode_operand(CUtensorMap *m, const void *base, int lk, int lrows, int lbat, long long nver, bool fp16,
                   bool fold = false, int box_rows = 128) {
    RC(get_encoder());
    cuuint64_t dims[4] = {(cuuint64_t)1 << lk, (cuuint64_t)1 << lrows, (cuuint64_t)4 << lbat, (cuuint64_t)nver};
    cuuint64_t strides[3] = {((cuuint64_t)1 << lk) * 2, ((cuuint64_t)1 << (lk + lrows)) * 2,
                             ((cuuint64_t)1 << (lk + lrows + lbat)) * 8};
    // folded: one box = all rows of box_rows >> lrows consecutive versions (box_rows rows)
    if (fold && lrows > __builtin_ctz((unsigned)box_rows)) {
        tn_set_error("encode_operand: folded operand wider than the tile");
        return TN_EINVAL;
    }
    cuuint32_t box[4] = {(cuuint32_t)tnk::kTcBK, fold ? (cuuint32_t)1 << lrows : (cuuint32_t)box_rows, 1,
                         fold ? (cuuint32_t)(box_rows >> lrows) : 1u};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = g_encode(m, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                          const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        tn_set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return TN_EDEVICE;
    }
    return TN_OK;
}

int setup_leaves(DevMem &mem, CNet &cn) {
    const int L = (int)cn.net.leaves.size();
    if (!cn.err.p) {
        RC(ensure(mem, cn.err, sizeof(int)));
        CK(cudaMemsetAsync(cn.err.p, 0, sizeof(int), mem.stream));
        cn.d_err = static_cast<int *>(cn.err.p);
    }
    static bool smem_set = false;
    if (!smem_set) {
        CK(cudaFuncSetAttribute(tnk::tc_cgemm<128, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tnk::TcSmem<128, 3>::kBytes));
        CK(cudaFuncSetAttribute(tnk::tc_cgemm<64, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tnk::TcSmem<64, 4>::kBytes));
        CK(cudaFuncSetAttribute(tnk::tc_cgemm<32, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tnk::TcSmem<32, 5>::kBytes));
        CK(cudaFuncSetAttribute(tnk::tc_stack_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                8 << kStackMaxBeta));
        smem_set = true;
    }
    for (auto &b : cn.leaf_src) release(mem, b);
    for (auto &b : cn.leaf_dst) release(mem, b);
    cn.leaf_src.assign(L, DBuf());
    cn.leaf_dst.assign(L, DBuf());
    cn.leaf_codebits.assign(L, 0);
    cn.leaf_sl.assign(L, {});
    std::vector<tnk::MatDesc> static_descs;
    cn.leaf_bytes = 0;
    for (int i = 0; i < L; i++) {
        const Leaf &lf = cn.net.leaves[i];
        const Node &nd = cn.tree.nodes[i];
        tnk::MatDesc d;
        std::memset(&d, 0, sizeof(d));
        std::vector<int> sl;
        for (size_t l = 0; l < lf.kind.size(); l++)
            if (lf.kind[l] == LEG_SLICED && ((cn.E >> lf.ref[l]) & 1)) { sl.push_back((int)l); cn.leaf_sl[i].push_back(lf.ref[l]); }
        if (sl.size() > 8 || nd.layout.size() > (size_t)tnk::kMaxBits) {
            tn_set_error("leaf with too many legs");
            return TN_EUNSUPPORTED;
        }
        d.nd = (int)nd.layout.size();
        d.ncode_bits = (int)sl.size();
        for (int t = 0; t < d.nd; t++) {
            int id = nd.layout[t];
            int leg = -1;
            const bool vbit = id >= cn.net.n_idx && id < cn.net.n_idx + cn.net.n_sliced;
            for (size_t l = 0; l < lf.kind.size(); l++) {
                if (lf.kind[l] == LEG_NET && lf.ref[l] == id) leg = (int)l;
                if (vbit && lf.kind[l] == LEG_SLICED && lf.ref[l] == id - cn.net.n_idx) leg = (int)l;
            }
            if (leg >= 0) d.dst_leg[t] = (int8_t)leg;
            else { tn_set_error("leaf layout index not found"); return TN_EINVAL; }
        }
        for (size_t u = 0; u < sl.size(); u++) d.sl_leg[u] = (int8_t)sl[u];
        cn.leaf_codebits[i] = d.ncode_bits;
        size_t src_bytes = lf.data.size() * sizeof(double2);
        RC(ensure(mem, cn.leaf_src[i], src_bytes));
        CK(cudaMemcpyAsync(cn.leaf_src[i].p, lf.data.data(), src_bytes, cudaMemcpyHostToDevice, mem.stream));
        size_t dst_bytes = (size_t(1) << (d.nd + d.ncode_bits)) * cn.elem;
        RC(ensure(mem, cn.leaf_dst[i], dst_bytes));
        cn.leaf_bytes += dst_bytes + src_bytes;
        d.src = static_cast<const double2 *>(cn.leaf_src[i].p);
        d.dst = cn.leaf_dst[i].p;
        d.fmt = cn.elem == 8 ? cn.fmt[i] : tnk::OUT_C64;
        d.scale = cn.scale[i];
        static_descs.push_back(d);
    }
    // leaves are materialised once per compiled variant and format assignment
    if (!static_descs.empty()) {
        ScopedBuf tmp(mem);
        RC(ensure(mem, tmp.b, static_descs.size() * sizeof(tnk::MatDesc)));
        CK(cudaMemcpyAsync(tmp.b.p, static_descs.data(), static_descs.size() * sizeof(tnk::MatDesc),
                           cudaMemcpyHostToDevice, mem.stream));
        dim3 grid(4, (unsigned)static_descs.size());
        if (cn.elem == 8) tnk::materialize<float2><<<grid, 256, 0, mem.stream>>>((const tnk::MatDesc *)tmp.b.p);
        else tnk::materialize<double2><<<grid, 256, 0, mem.stream>>>((const tnk::MatDesc *)tmp.b.p);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(mem.stream));
    }
    cn.cp.valid = false;
    CK(cudaStreamSynchronize(mem.stream));
    cn.parent.assign(cn.tree.nodes.size(), -1);
    for (size_t i = 0; i < cn.tree.nodes.size(); i++)
        for (int c : cn.tree.nodes[i].ch)
            if (c >= 0) cn.parent[c] = (int)i;
    return TN_OK;
}

void drop_graphs(CNet &cn) {
    for (int i = 0; i < 2; i++)
        if (cn.graph[i]) {
            cudaGraphExecDestroy(cn.graph[i]);
            cn.graph[i] = nullptr;
        }
}

void free_cnet(DevMem &mem, CNet &cn) {
    drop_graphs(cn);
    for (auto &b : cn.leaf_src) release(mem, b);
    for (auto &b : cn.leaf_dst) release(mem, b);
    release(mem, cn.gdescs);
    release(mem, cn.gtabs);
    release(mem, cn.arena);
    release(mem, cn.tables);
    release(mem, cn.vidx_dev);
    release(mem, cn.stacks);
    release(mem, cn.err);
    release(mem, cn.absmax);
    cn.d_err = nullptr;
    for (auto &x : cn.ev) cudaEventDestroy(x);
    cn.ev.clear();
}

inline uint64_t leaf_code(uint64_t w, const std::vector<int> &sl) {
    uint64_t code = 0;
    for (size_t u = 0; u < sl.size(); u++) code |= ((w >> sl[u]) & 1ull) << u;
    return code;
}

// Versions, arena offsets and pointer tables for a slice set.
int prepare_call(DevMem &mem, CNet &cn, const std::vector<uint64_t> &slices, double budget) {
    if (cn.cp.valid && cn.cp.slices == slices) return TN_OK;
    drop_graphs(cn);
    CallPlan cp;
    cp.slices = slices;
    const auto &nodes = cn.tree.nodes;
    CallLayout lay;
    layout_call(cn.tree, cn.steps, cn.E, cn.elem, slices, lay);
    auto &vals = lay.vals;
    auto &index = lay.index;
    cp.nver = lay.nver;
    // tensor-core steps at call time: a step whose per-version rows (or columns) are too
    // few is folded when the other operand is shared by all versions and this operand's
    // versions are consecutive: the versions stack into one M (or N) axis
    cp.fold.assign(cn.steps.size(), 0);
    if (cn.elem == 8 && cn.prec != TN_PREC_C64) {
        std::vector<char> u(cn.steps.size(), 0);
        auto vindex = [&](int x, uint64_t w) -> long long {
            if (nodes[x].ch[0] < 0) return (long long)leaf_code(w, cn.leaf_sl[x]);
            return index[x].at(w);
        };
        for (size_t i = 0; i < cn.steps.size(); i++) {
            const Step &s = cn.steps[i];
            if (tc_step(s)) { u[i] = 1; continue; }
            const long long nv = cp.nver[s.c];
            if (s.nk < 4 || nv < 2) continue;
            const uint64_t Da = nodes[s.a].dep & cn.E, Db = nodes[s.b].dep & cn.E;
            bool a_const = true, b_const = true, a_seq = true, b_seq = true;
            const long long a0 = vindex(s.a, vals[s.c][0] & Da), b0 = vindex(s.b, vals[s.c][0] & Db);
            for (long long v = 0; v < nv; v++) {
                const long long ia = vindex(s.a, vals[s.c][v] & Da), ib = vindex(s.b, vals[s.c][v] & Db);
                a_const &= ia == a0;
                b_const &= ib == b0;
                a_seq &= ia == a0 + v;
                b_seq &= ib == b0 + v;
            }
            if (s.nm < 7 && s.nn >= 6 && b_const && a_seq && (nv << s.nm) >= 64) { u[i] = 1; cp.fold[i] = 1; }
            else if (s.nn < 7 && s.nm >= 6 && a_const && b_seq && (nv << s.nn) >= 64) { u[i] = 1; cp.fold[i] = 2; }
        }
        if (u != cn.use_tc) {
            apply_formats(cn, u);
            drop_graphs(cn);
            RC(setup_leaves(mem, cn));
        }
    }
    cp.off = lay.off;
    cp.arena_bytes = lay.arena_bytes;
    if ((double)cp.arena_bytes + (double)cn.leaf_bytes > budget) {
        tn_set_error("working set of " + std::to_string(cp.arena_bytes) + " bytes exceeds the HBM budget");
        return TN_ENOMEM;
    }
    RC(ensure(mem, cn.arena, cp.arena_bytes));
    // pointer tables
    auto base_of = [&](int x, uint64_t w) -> const void * {
        if (nodes[x].ch[0] < 0) {
            uint64_t code = leaf_code(w, cn.leaf_sl[x]);
            size_t sz = (size_t(1) << nodes[x].layout.size()) * cn.elem;
            return static_cast<const char *>(cn.leaf_dst[x].p) + code * sz;
        }
        size_t sz = (size_t(1) << nodes[x].layout.size()) * cn.elem;
        return static_cast<const char *>(cn.arena.p) + cp.off[x] + (size_t)index[x].at(w) * sz;
    };
    cp.host_tab.clear();
    cp.tab_off.clear();
    cp.flops_all = lay.flops;
    cp.flops_beta = lay.flops_beta;
    cp.goff = lay.goff;
    auto version_index = [&](int x, uint64_t w) -> int {
        if (nodes[x].ch[0] < 0) return (int)leaf_code(w, cn.leaf_sl[x]);
        return index[x].at(w);
    };
    // operand o of step i: its own storage, or the step's gathered copy
    auto operand_base = [&](size_t i, int o, uint64_t w) -> const void * {
        const Step &s = cn.steps[i];
        const int x = o ? s.b : s.a;
        if (!s.gat[o]) return base_of(x, w);
        const size_t sz = (size_t(1) << s.g_nbits[o]) * cn.elem;
        return static_cast<const char *>(cn.arena.p) + cp.goff[i][o] + (size_t)version_index(x, w) * sz;
    };
    for (size_t i = 0; i < cn.steps.size(); i++) {
        const Step &s = cn.steps[i];
        cp.tab_off.push_back(cp.host_tab.size());
        const uint64_t Da = nodes[s.a].dep & cn.E, Db = nodes[s.b].dep & cn.E;
        for (uint64_t w : vals[s.c]) cp.host_tab.push_back(operand_base(i, 0, w & Da));
        for (uint64_t w : vals[s.c]) cp.host_tab.push_back(operand_base(i, 1, w & Db));
    }
    cp.root_tab = cp.host_tab.size();
    const int root = cn.tree.root;
    for (uint64_t w : vals[root]) cp.host_tab.push_back(base_of(root, w));
    cp.root_nver = (long long)vals[root].size();
    // tensor-core steps: one 4-D map per operand over all its versions (leaf codes or
    // the node's arena versions) and a table giving each C version's operand versions
    cp.map_off.assign(cn.steps.size(), 0);
    cp.vidx_off.assign(cn.steps.size(), 0);
    cp.tc_inplace.assign(cn.steps.size(), {0, 0});
    cp.maps.clear();
    cp.vidx.clear();
    auto version_count = [&](int x) -> long long {
        if (nodes[x].ch[0] < 0) return 1LL << cn.leaf_sl[x].size();
        return cp.nver[x];
    };
    auto region = [&](int x) -> const void * {
        if (nodes[x].ch[0] < 0) return cn.leaf_dst[x].p;
        return static_cast<const char *>(cn.arena.p) + cp.off[x];
    };
    for (size_t i = 0; i < cn.steps.size(); i++) {
        if (cn.use_tc.empty() || !cn.use_tc[i]) continue;
        const Step &s = cn.steps[i];
        cp.map_off[i] = cp.maps.size();
        cp.vidx_off[i] = cp.vidx.size();
        const bool f16 = cn.fmt[s.a] == tnk::OUT_SPLIT_FP16;
        CUtensorMap ma, mb;
        // a gathered operand of an unfolded step is read in place: its map spans the stored
        // form, whose batch planes are the non-beta batch bits and the closed legs on top
        const int nnb = s.nbat - cn.net.n_beta;
        const bool ipa = s.gat[0] && cp.fold[i] == 0 && nnb >= 0, ipb = s.gat[1] && cp.fold[i] == 0 && nnb >= 0;
        cp.tc_inplace[i] = {(char)ipa, (char)ipb};
        const void *ra = ipa ? region(s.a) : s.gat[0] ? static_cast<const char *>(cn.arena.p) + cp.goff[i][0]
                                                      : region(s.a);
        const void *rb = ipb ? region(s.b) : s.gat[1] ? static_cast<const char *>(cn.arena.p) + cp.goff[i][1]
                                                      : region(s.b);
        const int lba = ipa ? nnb + s.g_nq[0] : s.nbat, lbb = ipb ? nnb + s.g_nq[1] : s.nbat;
        // B for 128-, 64- and 32-column tiles (a folded B wider than a tile keeps the
        // 128-column map; those variants are not offered for it)
        CUtensorMap mb64, mb32;
        RC(encode_operand(&ma, ra, s.nk, s.nm, lba, version_count(s.a), f16, cp.fold[i] == 1));
        RC(encode_operand(&mb, rb, s.nk, s.nn, lbb, version_count(s.b), f16, cp.fold[i] == 2));
        if (cp.fold[i] == 2 && s.nn > 6) mb64 = mb;
        else RC(encode_operand(&mb64, rb, s.nk, s.nn, lbb, version_count(s.b), f16, cp.fold[i] == 2, 64));
        if (cp.fold[i] == 2 && s.nn > 5) mb32 = mb;
        else RC(encode_operand(&mb32, rb, s.nk, s.nn, lbb, version_count(s.b), f16, cp.fold[i] == 2, 32));
        cp.maps.push_back(ma);
        cp.maps.push_back(mb);
        cp.maps.push_back(mb64);
        cp.maps.push_back(mb32);
        const uint64_t Da = nodes[s.a].dep & cn.E, Db = nodes[s.b].dep & cn.E;
        for (uint64_t w : vals[s.c]) cp.vidx.push_back(version_index(s.a, w & Da));
        for (uint64_t w : vals[s.c]) cp.vidx.push_back(version_index(s.b, w & Db));
    }
    // batch gathers: one descriptor per gathered operand, grouped by step
    cp.gd.clear();
    cp.gd_off.assign(cn.steps.size() + 1, 0);
    for (size_t i = 0; i < cn.steps.size(); i++) {
        cp.gd_off[i] = cp.gd.size();
        const Step &s = cn.steps[i];
        for (int o = 0; o < 2; o++) {
            if (!s.gat[o]) continue;
            const int x = o ? s.b : s.a;
            tnk::GatherDesc g;
            std::memset(&g, 0, sizeof(g));
            g.src = static_cast<const char *>(region(x));
            g.dst = static_cast<char *>(cn.arena.p) + cp.goff[i][o];
            g.nver = version_count(x);
            const bool split = cn.elem == 8 && cn.fmt[x] != tnk::OUT_C64;
            g.nplanes = split ? 4 : 1;
            g.esize = split ? 2 : cn.elem;
            g.src_plane = 1LL << nodes[x].layout.size();
            g.dst_plane = 1LL << s.g_nbits[o];
            g.nbits = s.g_nbits[o];
            g.lb = cn.net.n_beta;
            g.nq = s.g_nq[o];
            std::vector<std::pair<int, int>> pb;
            for (int t = 0; t < g.lb; t++) pb.push_back({s.g_pos_beta[o][t], t});
            std::sort(pb.rbegin(), pb.rend());
            int lowrun = g.nbits;
            for (int t = 0; t < g.lb; t++) {
                g.pos_beta[t] = (int8_t)pb[t].first;
                g.beta_bit[t] = (int8_t)pb[t].second;
                lowrun = std::min(lowrun, pb[t].first);
            }
            for (int q = 0; q < g.nq; q++) g.q[q] = s.g_q[o][q];
            const int vw = g.esize == 2 ? 3 : g.esize == 8 ? 1 : 0;
            g.vec_log2 = lowrun >= vw ? vw : 0;
            g.run_log2 = lowrun - g.vec_log2;
            if (g.src_plane != 1LL << (g.nbits - g.lb + g.nq)) {
                tn_set_error("gather: stored operand size does not match its read layout");
                return TN_EINVAL;
            }
            cp.gd.push_back(g);
        }
    }
    cp.gd_off[cn.steps.size()] = cp.gd.size();
    if (!cp.gd.empty()) {
        // byte lookup tables of every gather's bit maps (see tnk::GatherDesc)
        const size_t W = tnk::kGatherTabWords;
        cp.gtab.assign(cp.gd.size() * W, 0ull);
        RC(ensure(mem, cn.gtabs, cp.gtab.size() * sizeof(uint64_t)));
        for (size_t gi = 0; gi < cp.gd.size(); gi++) {
            tnk::GatherDesc &g = cp.gd[gi];
            uint64_t *rest = cp.gtab.data() + gi * W;
            uint32_t *beta = reinterpret_cast<uint32_t *>(rest + 5 * 256), *sel = beta + 5 * 256;
            tn_gather_tables(g.nbits, g.lb, g.pos_beta, g.beta_bit, g.nq, g.q, rest, beta, sel);
            const uint64_t *dev = static_cast<const uint64_t *>(cn.gtabs.p) + gi * W;
            g.rest_tab = dev;
            g.beta_tab = reinterpret_cast<const uint32_t *>(dev + 5 * 256);
            g.sel_tab = g.beta_tab + 5 * 256;
        }
        CK(cudaMemcpyAsync(cn.gtabs.p, cp.gtab.data(), cp.gtab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice,
                           mem.stream));
        RC(ensure(mem, cn.gdescs, cp.gd.size() * sizeof(tnk::GatherDesc)));
        CK(cudaMemcpyAsync(cn.gdescs.p, cp.gd.data(), cp.gd.size() * sizeof(tnk::GatherDesc), cudaMemcpyHostToDevice,
                           mem.stream));
    }
    // the stack list of stacked tensor-core tiles (any step with an in-place A may use them)
    for (size_t i = 0; i < cn.steps.size(); i++) {
        if (!cp.tc_inplace[i][0] || cn.net.n_beta > kStackMaxBeta) continue;
        RC(ensure(mem, cn.stacks, (1 + ((size_t)(tnk::kTcMaxStack + 1) << cn.net.n_beta)) * sizeof(int)));
        break;
    }
    if (!cp.vidx.empty()) {
        RC(ensure(mem, cn.vidx_dev, cp.vidx.size() * sizeof(int)));
        CK(cudaMemcpyAsync(cn.vidx_dev.p, cp.vidx.data(), cp.vidx.size() * sizeof(int), cudaMemcpyHostToDevice,
                           mem.stream));
        CK(cudaStreamSynchronize(mem.stream));
    }
    RC(ensure(mem, cn.tables, cp.host_tab.size() * sizeof(void *)));
    CK(cudaMemcpyAsync(cn.tables.p, cp.host_tab.data(), cp.host_tab.size() * sizeof(void *),
                       cudaMemcpyHostToDevice, mem.stream));
    CK(cudaStreamSynchronize(mem.stream));
    cp.valid = true;
    cn.cp = std::move(cp);
    cn.variant.assign(cn.steps.size(), -1);
    return TN_OK;
}

// Kernel variants of a step (ids as in tn_step_trace.kernel): 0 row kernel, 1 staged
// small products, 4 staged row kernel, 5 long-K kernel, TM*1000+TN FFMA tile, 9128 / 9064 /
// 9032 tensor-core tile of 128 / 64 / 32 columns, 19128 / 19064 stacked tensor-core tile of
// 128 / 64 columns (batches sharing a stored block of A side by side).
constexpr int kVarRow = 0, kVarSmall = 1, kVarRowStage = 4, kVarSkinny = 5, kVarTc128 = 9128, kVarTc64 = 9064,
              kVarTc32 = 9032, kVarTcS128 = 19128, kVarTcS64 = 19064;

bool is_tc_variant(int v) {
    return v == kVarTc128 || v == kVarTc64 || v == kVarTc32 || v == kVarTcS128 || v == kVarTcS64;
}

// Whether step si can run stacked tensor-core tiles of BN columns: A read in place from its
// stored form, N of 32 or 64 (two to four batches per tile), at most 2^14 batches per
// group, and a B read in place (if any) with its batch-index bits where A has them.
bool stack_fits(const CNet &cn, size_t si, int BN) {
    const Step &s = cn.steps[si];
    const CallPlan &cp = cn.cp;
    if (cn.use_tc.empty() || !cn.use_tc[si] || cp.tc_inplace.size() <= si || !cp.tc_inplace[si][0]) return false;
    if (!cn.stacks.p || cp.fold.size() <= si || cp.fold[si] != 0) return false;
    if ((s.nn != 5 && s.nn != 6) || (BN >> s.nn) < 2 || (BN >> s.nn) > tnk::kTcMaxStack) return false;
    const int nb = cn.net.n_beta;
    if (nb < 1 || nb > kStackMaxBeta || s.nbat < nb || s.nbat > 24) return false;
    if (cp.tc_inplace[si][1])
        for (int t = 0; t < nb; t++)
            if (s.g_pos_beta[1][t] - (s.nk + s.nn) != s.g_pos_beta[0][t] - (s.nk + s.nm)) return false;
    return true;
}

// Whether the staged row kernel can run step si: the row kernel's shapes with complex64
// rows of 16 to 64 elements.
bool rowstage_fits(const CNet &cn, const Step &s) {
    return cn.elem == 8 && std::min(s.nm, s.nn) <= 5 && s.nk >= 4 && s.nk <= 6;
}
constexpr int kTiles[7][2] = {{128, 64}, {64, 64}, {128, 32}, {64, 32}, {32, 32}, {128, 16}, {16, 16}};

// Whether the long-K kernel runs step si: at most 8 outputs on the short side and 64 on
// the long side, K >= 1024, complex64 operands.  It is then the step's only kernel (its
// lane split of K rounds differently from the others).
bool skinny_fits(const CNet &cn, const Step &s) {
    return cn.elem == 8 && std::min(s.nm, s.nn) <= 3 && std::max(s.nm, s.nn) <= 6 && s.nk >= 10 &&
           cn.fmt[s.a] == tnk::OUT_C64 && cn.fmt[s.b] == tnk::OUT_C64 &&
           (cn.use_tc.empty() || !cn.use_tc[&s - cn.steps.data()]);
}

bool small_fits(const Step &s, size_t esz) {
    return s.nm <= 6 && s.nn <= 6 && s.nk <= 6 && s.nbat >= 4 &&
           (size_t)(((1 << s.nm) + (1 << s.nn)) * ((1 << s.nk) + 1)) * esz <= 48 * 1024;
}

// Every variant that can run step si (the tensor-core ones when its operands are split).
std::vector<int> step_variants(const CNet &cn, size_t si) {
    const Step &s = cn.steps[si];
    std::vector<int> v;
    if (skinny_fits(cn, s)) return {kVarSkinny};
    if (!cn.use_tc.empty() && cn.use_tc[si]) {
        if (s.nn <= 5) v = {kVarTc32, kVarTc64};
        else if (s.nn == 6) v = {kVarTc128, kVarTc64, kVarTc32};
        else v = {kVarTc128, kVarTc64};
        if (stack_fits(cn, si, 128)) v.push_back(kVarTcS128);
        if (stack_fits(cn, si, 64)) v.push_back(kVarTcS64);
        return v;
    }
    if (std::min(s.nm, s.nn) <= 5 && s.nk <= 6) v.push_back(kVarRow);
    if (rowstage_fits(cn, s)) v.push_back(kVarRowStage);
    if (small_fits(s, (size_t)cn.elem)) v.push_back(kVarSmall);
    for (auto &t : kTiles)
        if (t[0] == 16 || ((2LL << s.nm) >= t[0] && (2LL << s.nn) >= t[1])) v.push_back(t[0] * 1000 + t[1]);
    return v;
}

// The fixed shape rules used without autotuning.
int default_variant(const CNet &cn, size_t si) {
    const Step &s = cn.steps[si];
    if (skinny_fits(cn, s)) return kVarSkinny;
    if (!cn.use_tc.empty() && cn.use_tc[si]) {
        // stacked tiles where they fit and the step is large enough to amortise building
        // the stack list (tens of microseconds)
        if (stack_fits(cn, si, 128) && s.flops_per_version * (double)cn.cp.nver[s.c] >= 1e9) return kVarTcS128;
        return s.nn <= 5 ? kVarTc32 : kVarTc128;
    }
    if (std::min(s.nm, s.nn) == 6 && std::max(s.nm, s.nn) == 6 && small_fits(s, (size_t)cn.elem)) return kVarSmall;
    if (std::min(s.nm, s.nn) <= 5 && s.nk <= 6) return kVarRow;
    // large products: 128 x 32 tiles (the autotuner's choice on GB300 for complex64)
    if (s.nm >= 7 && s.nn >= 5) return 128032;
    if (s.nm >= 6 && s.nn >= 6) return 64064;
    if (s.nm >= 6 && s.nn >= 5) return 64032;
    if (s.nm >= 5 && s.nn >= 5) return 32032;
    if (s.nm >= 7) return 128016;
    return 16016;
}

// The row kernel reads every gathered operand of step si through its gather (no copy)
// when each one is a single complex version whose batch bits lie above the span the
// kernel reads contiguously: a row (K) for the row operand, a batch's block (N x K) for
// the other.  `swap` says whether the kernel exchanges the roles (the longer side rows).
bool row_fuses(const CNet &cn, size_t si) {
    const Step &s = cn.steps[si];
    if (!(s.gat[0] || s.gat[1]) || cn.cp.gd_off.size() <= si + 1) return false;
    const bool swap = s.nn > s.nm;
    for (int o = 0; o < 2; o++) {
        if (!s.gat[o]) continue;
        const tnk::GatherDesc &g = cn.cp.gd[cn.cp.gd_off[si] + (o == 1 && s.gat[0] ? 1 : 0)];
        if (g.nver != 1 || g.nplanes != 1 || g.esize != cn.elem || g.lb < 1) return false;
        const int lowrun = g.pos_beta[g.lb - 1];
        const bool is_rows = (o == 0) != swap;  // this operand plays the kernel's A (rows)
        const int need = is_rows ? s.nk : s.nk + (swap ? s.nm : s.nn);
        if (lowrun < need) return false;
    }
    return true;
}

// The long-K kernel reads a gathered operand in place when it is a single complex version
// whose every row (K elements) is contiguous in its source.
bool skinny_fuses(const CNet &cn, size_t si) {
    const Step &s = cn.steps[si];
    if (!(s.gat[0] || s.gat[1]) || cn.cp.gd_off.size() <= si + 1) return false;
    for (int o = 0; o < 2; o++) {
        if (!s.gat[o]) continue;
        const tnk::GatherDesc &g = cn.cp.gd[cn.cp.gd_off[si] + (o == 1 && s.gat[0] ? 1 : 0)];
        if (g.nver != 1 || g.nplanes != 1 || g.esize != cn.elem || g.lb < 1) return false;
        if (g.pos_beta[g.lb - 1] < s.nk) return false;
    }
    return true;
}

// Whether variant var of step si reads its gathered operands in place (no gather launch).
bool reads_in_place(const CNet &cn, size_t si, int var) {
    if (var == kVarRow || var == kVarRowStage) return row_fuses(cn, si);
    if (var == kVarSkinny) return skinny_fuses(cn, si);
    if (is_tc_variant(var)) {
        const Step &s = cn.steps[si];
        if (!(s.gat[0] || s.gat[1]) || cn.cp.tc_inplace.size() <= si) return false;
        return (!s.gat[0] || cn.cp.tc_inplace[si][0]) && (!s.gat[1] || cn.cp.tc_inplace[si][1]);
    }
    return false;
}

template <int BN, int ST>
int launch_tc(CNet &cn, const Step &s, size_t si, const tnk::GemmParams &p, cudaStream_t st, bool stacked = false) {
    const CallPlan &cp = cn.cp;
    tnk::TcParams tp;
    std::memset(&tp, 0, sizeof(tp));
    tp.lm = s.nm;
    tp.ln = s.nn;
    tp.lk = s.nk;
    tp.lbat = s.nbat;
    tp.out_fmt = p.out_fmt;
    tp.in_fp16 = cn.fmt[s.a] == tnk::OUT_SPLIT_FP16;
    tp.out_scale = p.out_scale;
    tp.err = cn.d_err;
    tp.stall_cycles = cn.tc_stall;
    for (int o = 0; o < 2; o++) {
        if (cp.tc_inplace.size() <= si || !cp.tc_inplace[si][o]) continue;
        if (!cn.cur_closed) { tn_set_error("tensor-core step: batch patterns missing"); return TN_EINVAL; }
        tnk::TcGather &g = o ? tp.gb : tp.ga;
        const int base = s.nk + (o ? s.nn : s.nm);  // read-layout position of batch bit 0
        g.closed = cn.cur_closed;
        g.nnb = s.nbat - cn.net.n_beta;
        g.nq = s.g_nq[o];
        if (s.nbat > 24 || g.nq > 32) { tn_set_error("tensor-core gather too wide"); return TN_EUNSUPPORTED; }
        for (int t = 0; t < cn.net.n_beta; t++) {
            const int i = s.g_pos_beta[o][t] - base;
            if (i < 0 || i >= s.nbat) { tn_set_error("tensor-core gather: beta bit outside the batch dims"); return TN_EINVAL; }
            g.beta_mask |= 1u << i;
            g.beta_t[i] = (int8_t)t;
        }
        for (int t = 0; t < g.nq; t++) g.q[t] = (int8_t)s.g_q[o][t];
    }
    // stacked tiles: this group's stack list first (same stream), then tiles of S batches
    if (stacked) {
        if (!stack_fits(cn, si, BN) || !cn.cur_closed) {
            tn_set_error("stacked tensor-core tile: step not eligible");
            return TN_EINVAL;
        }
        tp.stack = static_cast<const int *>(cn.stacks.p);
        tp.stack_S = BN >> s.nn;
        tnk::tc_stack_build<<<1, 1024, (size_t)8 << cn.net.n_beta, st>>>(tp.ga, cn.net.n_beta, tp.stack_S,
                                                                          static_cast<int *>(cn.stacks.p));
        CK(cudaGetLastError());
    }
    tp.c_plane = p.c_vstride;
    for (int i = 0; i < s.nbat; i++) tp.pos_bat[i] = s.pos_bat[i];
    for (int i = 0; i < s.nm; i++) tp.pos_m[i] = s.pos_m[i];
    for (int i = 0; i < s.nn; i++) tp.pos_n[i] = s.pos_n[i];
    using Lay = tnk::TcSmem<BN, ST>;
    const int fold = cp.fold.empty() ? 0 : cp.fold[si];
    const int lbn = __builtin_ctz(BN);
    const int ltm = std::min(s.nm, 7), ltn = std::min(s.nn, lbn);
    long long tiles_m = 1LL << (s.nm - ltm), tiles_n = 1LL << (s.nn - ltn), tiles_v = p.nver;
    if (fold == 1) { const long long vm = 128 >> s.nm; tiles_m = (p.nver + vm - 1) / vm; tiles_v = 1; }
    if (fold == 2) {
        if (s.nn > lbn) { tn_set_error("tensor-core tile narrower than a folded operand"); return TN_EINVAL; }
        const long long vn = BN >> s.nn;
        tiles_n = (p.nver + vn - 1) / vn;
        tiles_v = 1;
    }
    const long long tiles = (tiles_m * tiles_n << s.nbat) * tiles_v;
    const long long blocks = std::min<long long>(tiles, num_sms());
    tp.C = p.C;
    tp.nver = (int)p.nver;
    tp.fold = fold;
    tp.vidx = static_cast<const int *>(cn.vidx_dev.p) + cp.vidx_off[si];
    // raster groups: the A panels of one group (128 rows x K, 8 bytes per element over
    // the four planes) stay within about 48 MB of L2 while the group sweeps the n tiles
    {
        const double panel = 128.0 * std::ldexp(1.0, s.nk) * 8.0;
        long long g = (long long)std::floor(48.0 * (1 << 20) / panel);
        tp.group_m = (int)std::max<long long>(1, std::min<long long>({g, 64, tiles_m}));
    }
    const CUtensorMap *m = &cp.maps[cp.map_off[si]];
    // B map: box of BN rows, or of one stacked batch's N rows
    const int ib = stacked ? (s.nn == 6 ? 2 : 3) : (BN == 128 ? 1 : BN == 64 ? 2 : 3);
    tnk::tc_cgemm<BN, ST><<<(unsigned)blocks, tnk::kTcThreads, Lay::kBytes, st>>>(m[0], m[ib], tp);
    CK(cudaGetLastError());
    return TN_OK;
}


// The launch parameters every kernel variant of step s starts from.
int step_params(const CNet &cn, const Step &s, tnk::GemmParams &p) {
    const CallPlan &cp = cn.cp;
    const auto &nodes = cn.tree.nodes;
    std::memset(&p, 0, sizeof(p));
    const void *const *tab = static_cast<const void *const *>(cn.tables.p);
    p.ptrA = tab + cp.tab_off[&s - cn.steps.data()];
    p.nver = cp.nver[s.c];
    p.ptrB = p.ptrA + p.nver;
    p.C = static_cast<char *>(cn.arena.p) + cp.off[s.c];
    p.c_vstride = 1LL << nodes[s.c].layout.size();
    p.lm = s.nm;
    p.ln = s.nn;
    p.lk = s.nk;
    p.lbat = s.nbat;
    if (s.nbat + s.nm + s.nn > tnk::kMaxBits) { tn_set_error("step too large"); return TN_EUNSUPPORTED; }
    for (int i = 0; i < s.nbat; i++) p.pos_bat[i] = s.pos_bat[i];
    for (int i = 0; i < s.nm; i++) p.pos_m[i] = s.pos_m[i];
    for (int i = 0; i < s.nn; i++) p.pos_n[i] = s.pos_n[i];
    p.out_fmt = cn.fmt[s.c];
    p.out_scale = cn.scale[s.c] / (cn.scale[s.a] * cn.scale[s.b]);
    p.err = cn.d_err;
    return TN_OK;
}

// The row kernel's roles: one thread per row of the larger side, the small side in
// registers (C = A B^T is symmetric in the operand roles); gathered operands read in
// place when possible.
void row_roles(const CNet &cn, const Step &s, tnk::GemmParams &p) {
    const size_t si = &s - cn.steps.data();
    if (row_fuses(cn, si) && cn.cur_closed) {
        const auto *gd = static_cast<const tnk::GatherDesc *>(cn.gdescs.p) + cn.cp.gd_off[si];
        p.gA = s.gat[0] ? gd : nullptr;
        p.gB = s.gat[1] ? gd + (s.gat[0] ? 1 : 0) : nullptr;
        p.closed_bits = cn.cur_closed;
    }
    if (s.nn > s.nm) {
        std::swap(p.ptrA, p.ptrB);
        std::swap(p.gA, p.gB);
        std::swap(p.lm, p.ln);
        for (int i = 0; i < tnk::kMaxBits; i++) std::swap(p.pos_m[i], p.pos_n[i]);
        p.swapped = 1;
    }
}

template <typename T>
int launch_variant(CNet &cn, const Step &s, cudaStream_t st, int var) {
    tnk::GemmParams p;
    RC(step_params(cn, s, p));
    const size_t si = &s - cn.steps.data();
    if (cn.trace) cn.tr_kernel[si] = var;
    if (is_tc_variant(var)) {
        if constexpr (sizeof(T) == sizeof(float2)) {
            if (var == kVarTc128) return launch_tc<128, 3>(cn, s, si, p, st);
            if (var == kVarTc64) return launch_tc<64, 4>(cn, s, si, p, st);
            if (var == kVarTcS128) return launch_tc<128, 3>(cn, s, si, p, st, true);
            if (var == kVarTcS64) return launch_tc<64, 4>(cn, s, si, p, st, true);
            return launch_tc<32, 5>(cn, s, si, p, st);
        }
        tn_set_error("tensor-core variant on a complex128 network");
        return TN_EINVAL;
    }
    if (var == kVarSmall) {
        // stage 2^lg batches per block in shared memory
        const int per = ((1 << s.nm) + (1 << s.nn)) * ((1 << s.nk) + 1);  // padded elements per batch
        int lg = 0;
        while (lg < s.nbat && (size_t)(per << (lg + 1)) * sizeof(T) <= 48 * 1024 && (1 << (lg + 1 + s.nm + s.nn)) <= 4096) lg++;
        tnk::SmallMap sm;
        std::memset(&sm, 0, sizeof(sm));
        sm.lg = lg;
        std::vector<std::pair<int, std::pair<int, int>>> bits;  // (C position, (kind, index))
        for (int i = 0; i < lg; i++) bits.push_back({s.pos_bat[i], {0, i}});
        for (int i = 0; i < s.nm; i++) bits.push_back({s.pos_m[i], {1, i}});
        for (int i = 0; i < s.nn; i++) bits.push_back({s.pos_n[i], {2, i}});
        std::sort(bits.begin(), bits.end());
        sm.nloc = (int)bits.size();
        for (int i = 0; i < sm.nloc; i++) {
            sm.kind[i] = (int8_t)bits[i].second.first;
            sm.idx[i] = (int8_t)bits[i].second.second;
        }
        const long long blocks = p.nver << (s.nbat - lg);
        const size_t smem = (size_t)(per << lg) * sizeof(T);
        tnk::cgemm_small<T><<<(unsigned)blocks, 256, smem, st>>>(p, sm);
    } else if (var == kVarRowStage) {
        if (!rowstage_fits(cn, s)) { tn_set_error("staged row kernel: unsupported step shape"); return TN_EINVAL; }
        if constexpr (sizeof(T) == sizeof(float2)) {
            row_roles(cn, s, p);
            const long long rows = p.nver << (p.lbat + p.lm);
            const int per_block = 32 * tnk::kRowWarps;
            const size_t smem = (size_t)per_block * (8 * (1 << p.lk) + tnk::kRowPad);
            const unsigned blocks = (unsigned)std::min<long long>((rows + per_block - 1) / per_block, 3LL * num_sms());
            auto go = [&](auto kern) -> int {
                CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                kern<<<blocks, per_block, smem, st>>>(p);
                return TN_OK;
            };
            switch (p.ln) {
                case 0: RC(go(tnk::cgemm_rowstage<1>)); break;
                case 1: RC(go(tnk::cgemm_rowstage<2>)); break;
                case 2: RC(go(tnk::cgemm_rowstage<4>)); break;
                case 3: RC(go(tnk::cgemm_rowstage<8>)); break;
                case 4: RC(go(tnk::cgemm_rowstage<16>)); break;
                default: RC(go(tnk::cgemm_rowstage<32>)); break;
            }
        }
    } else if (var == kVarSkinny) {
        if (!skinny_fits(cn, s)) { tn_set_error("long-K kernel: unsupported step shape"); return TN_EINVAL; }
        if constexpr (sizeof(T) == sizeof(float2)) {
            const size_t si2 = &s - cn.steps.data();
            if (cn.cur_closed && skinny_fuses(cn, si2)) {
                const auto *gd = static_cast<const tnk::GatherDesc *>(cn.gdescs.p) + cn.cp.gd_off[si2];
                p.gA = s.gat[0] ? gd : nullptr;
                p.gB = s.gat[1] ? gd + (s.gat[0] ? 1 : 0) : nullptr;
                p.closed_bits = cn.cur_closed;
            }
            // the longer side are the kernel's rows (C = A B^T is symmetric in the roles)
            if (p.ln > p.lm) {
                std::swap(p.ptrA, p.ptrB);
                std::swap(p.gA, p.gB);
                std::swap(p.lm, p.ln);
                for (int i = 0; i < tnk::kMaxBits; i++) std::swap(p.pos_m[i], p.pos_n[i]);
            }
            // blocks of W warps with MW rows of A each (W MW = min(M, 32) rows per block),
            // as many as fit at once (each streams its share of the units through its ring)
            const long long units = (p.nver << p.lbat) * std::max(1, (1 << p.lm) / 32);
            int rc_go = TN_OK;
            auto go = [&](auto kern, int warps, int stage_bytes) {
                const int smem = tnk::kSkinnyST * stage_bytes;
                int per_sm = 0;
                if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem) != cudaSuccess ||
                    per_sm < 1) {
                    tn_set_error("long-K kernel: launch configuration rejected");
                    rc_go = TN_EDEVICE;
                    return;
                }
                const unsigned blocks = (unsigned)std::min<long long>(units, (long long)per_sm * num_sms());
                kern<<<blocks, 32 * warps, smem, st>>>(p);
            };
            auto by_n = [&](auto m_tag) {
                constexpr int M = decltype(m_tag)::value;
                // two rows per warp: 32-row blocks get 16 warps, enough to keep the FMA pipe
                // fed (4096 batches of 64 x 8 outputs over K = 2048: 1.58 ms, against 2.0 ms
                // with 8 warps of four rows and 1.95 ms with 32 warps of one row)
                constexpr int W = M >= 2 ? M / 2 : 1, MW = M / W;
                switch (p.ln) {
                    case 0: go(tnk::cgemm_skinny<W, MW, 1>, W, tnk::skinny_stage_bytes<W, MW, 1>()); break;
                    case 1: go(tnk::cgemm_skinny<W, MW, 2>, W, tnk::skinny_stage_bytes<W, MW, 2>()); break;
                    case 2: go(tnk::cgemm_skinny<W, MW, 4>, W, tnk::skinny_stage_bytes<W, MW, 4>()); break;
                    default: go(tnk::cgemm_skinny<W, MW, 8>, W, tnk::skinny_stage_bytes<W, MW, 8>()); break;
                }
            };
            switch (p.lm) {
                case 0: by_n(std::integral_constant<int, 1>{}); break;
                case 1: by_n(std::integral_constant<int, 2>{}); break;
                case 2: by_n(std::integral_constant<int, 4>{}); break;
                case 3: by_n(std::integral_constant<int, 8>{}); break;
                case 4: by_n(std::integral_constant<int, 16>{}); break;
                default: by_n(std::integral_constant<int, 32>{}); break;  // 64 rows: two row blocks
            }
            if (rc_go != TN_OK) return rc_go;
        } else {
            tn_set_error("long-K kernel on a complex128 network");
            return TN_EINVAL;
        }
    } else if (var == kVarRow) {
        row_roles(cn, s, p);
        long long rows = p.nver << (p.lbat + p.lm);
        // grid-stride: at most 16 resident blocks' worth per SM, each thread several rows
        unsigned blocks = (unsigned)std::min<long long>((rows + 255) / 256, 16LL * num_sms());
        switch (p.ln) {
            case 0: tnk::cgemm_row<T, 1><<<blocks, 256, 0, st>>>(p); break;
            case 1: tnk::cgemm_row<T, 2><<<blocks, 256, 0, st>>>(p); break;
            case 2: tnk::cgemm_row<T, 4><<<blocks, 256, 0, st>>>(p); break;
            case 3: tnk::cgemm_row<T, 8><<<blocks, 256, 0, st>>>(p); break;
            case 4: tnk::cgemm_row<T, 16><<<blocks, 256, 0, st>>>(p); break;
            default: tnk::cgemm_row<T, 32><<<blocks, 256, 0, st>>>(p); break;
        }
    } else {
        auto launch = [&](auto kern, int TM, int TN) {
            int ltm = std::min(s.nm, __builtin_ctz(TM)), ltn = std::min(s.nn, __builtin_ctz(TN));
            long long blocks = p.nver << (s.nbat + (s.nm - ltm) + (s.nn - ltn));
            kern<<<(unsigned)blocks, 256, 0, st>>>(p);
        };
        constexpr int TK = sizeof(T) == 8 ? 16 : 8;
        switch (var) {
            case 128064: launch(tnk::cgemm_tile<T, 128, 64, TK, 8, 4>, 128, 64); break;
            case 64064: launch(tnk::cgemm_tile<T, 64, 64, TK, 4, 4>, 64, 64); break;
            case 128032: launch(tnk::cgemm_tile<T, 128, 32, TK, 8, 2>, 128, 32); break;
            case 64032: launch(tnk::cgemm_tile<T, 64, 32, TK, 4, 2>, 64, 32); break;
            case 32032: launch(tnk::cgemm_tile<T, 32, 32, TK, 2, 2>, 32, 32); break;
            case 128016: launch(tnk::cgemm_tile<T, 128, 16, TK, 4, 2>, 128, 16); break;
            case 16016: launch(tnk::cgemm_tile<T, 16, 16, TK, 1, 1>, 16, 16); break;
            default: tn_set_error("unknown kernel variant " + std::to_string(var)); return TN_EINVAL;
        }
    }
    CK(cudaGetLastError());
    return TN_OK;
}

template <typename T>
int launch_step(CNet &cn, const Step &s, cudaStream_t st) {
    const size_t si = &s - cn.steps.data();
    const int var = si < cn.variant.size() && cn.variant[si] >= 0 ? cn.variant[si] : default_variant(cn, si);
    return launch_variant<T>(cn, s, st, var);
}

int launch_gathers(CNet &cn, size_t si, const uint64_t *d_closed, cudaStream_t st) {
    const size_t ng = cn.cp.gd_off[si + 1] - cn.cp.gd_off[si];
    if (!ng) return TN_OK;
    if (!d_closed) { tn_set_error("execute: batch patterns missing"); return TN_EINVAL; }
    long long most = 0;
    for (size_t g = cn.cp.gd_off[si]; g < cn.cp.gd_off[si + 1]; g++) {
        const auto &d = cn.cp.gd[g];
        most = std::max(most, (d.dst_plane >> d.vec_log2) * d.nplanes * d.nver);
    }
    dim3 grid((unsigned)std::min<long long>((most + 255) / 256, 4 * num_sms()), (unsigned)ng);
    tnk::gather_batches<<<grid, 256, 0, st>>>(static_cast<const tnk::GatherDesc *>(cn.gdescs.p) + cn.cp.gd_off[si],
                                              d_closed);
    CK(cudaGetLastError());
    return TN_OK;
}

int launch_slice_sum(CNet &cn, double2 *out, cudaStream_t st) {
    const int root = cn.tree.root;
    const int nout = (int)cn.net.out_layout.size();
    const int nfree = (int)cn.tree.nodes[root].layout.size() - nout;
    long long nelem = 1LL << nout;
    const void *const *rt = static_cast<const void *const *>(cn.tables.p) + cn.cp.root_tab;
    unsigned blocks = (unsigned)((nelem + 255) / 256);
    const size_t ss = cn.steps.size();
    if (cn.trace) {
        if (cn.ev_pending[ss]) {
            float ms = 0;
            CK(cudaEventSynchronize(cn.ev[2 * ss + 1]));
            CK(cudaEventElapsedTime(&ms, cn.ev[2 * ss], cn.ev[2 * ss + 1]));
            cn.tr_ms[ss] += ms;
            cn.tr_launches[ss]++;
            cn.ev_pending[ss] = 0;
        }
        CK(cudaEventRecord(cn.ev[2 * ss], st));
    }
    if (cn.elem == 8) tnk::slice_sum<float2><<<blocks, 256, 0, st>>>(rt, cn.cp.root_nver, nfree, nout, out);
    else tnk::slice_sum<double2><<<blocks, 256, 0, st>>>(rt, cn.cp.root_nver, nfree, nout, out);
    CK(cudaGetLastError());
    if (cn.trace) {
        CK(cudaEventRecord(cn.ev[2 * ss + 1], st));
        cn.ev_pending[ss] = 1;
        cn.tr_kernel[ss] = 2;
    }
    return TN_OK;
}

// The root step's index when it runs fused with the slice sum (-1: not fused).  Fusion
// needs the row kernel on a root stored as plain complex values, batch, row and column
// bits that cover the root layout once each, and free patterns that fit the fused
// kernel's byte tables; it is off while FP16 scales are calibrated (every node's maximum
// is recorded from its stored values).
long long fused_root_step(const CNet &cn) {
    if (!cn.fuse_root || cn.calibrating || cn.steps.empty() || !cn.cp.valid) return -1;
    const int root = cn.tree.root;
    const size_t si = cn.steps.size() - 1;
    const Step &s = cn.steps[si];
    if (s.c != root) return -1;
    const int var = si < cn.variant.size() && cn.variant[si] >= 0 ? cn.variant[si] : default_variant(cn, si);
    if (var != kVarRow || cn.fmt[root] != tnk::OUT_C64) return -1;
    const int nout = (int)cn.net.out_layout.size();
    const int nfree = (int)cn.tree.nodes[root].layout.size() - nout;
    if (nfree < 0 || nfree > 8 * tnk::kRootTabBytes || cn.cp.nver[root] != cn.cp.root_nver) return -1;
    if (s.nbat + s.nm + s.nn != nout + nfree || nout + nfree > tnk::kMaxBits) return -1;
    uint64_t seen = 0;
    auto mark = [&](const int8_t *pos, int n) {
        for (int i = 0; i < n; i++) {
            if (pos[i] < 0 || pos[i] >= nout + nfree || ((seen >> pos[i]) & 1)) return false;
            seen |= 1ull << pos[i];
        }
        return true;
    };
    if (!mark(s.pos_bat, s.nbat) || !mark(s.pos_m, s.nm) || !mark(s.pos_n, s.nn)) return -1;
    return (long long)si;
}

// The root step (row kernel) and the FP64 slice sum in one launch: bit-identical to the
// two launched one after the other, without the root's values passing through memory.
int launch_root_slice_sum(CNet &cn, size_t si, double2 *out, cudaStream_t st) {
    const int root = cn.tree.root;
    const int nout = (int)cn.net.out_layout.size();
    const int nfree = (int)cn.tree.nodes[root].layout.size() - nout;
    tnk::GemmParams p;
    RC(step_params(cn, cn.steps[si], p));
    row_roles(cn, cn.steps[si], p);
    const size_t ss = cn.steps.size();
    if (cn.trace) {
        if (cn.ev_pending[ss]) {
            float ms = 0;
            CK(cudaEventSynchronize(cn.ev[2 * ss + 1]));
            CK(cudaEventElapsedTime(&ms, cn.ev[2 * ss], cn.ev[2 * ss + 1]));
            cn.tr_ms[ss] += ms;
            cn.tr_launches[ss]++;
            cn.ev_pending[ss] = 0;
        }
        CK(cudaEventRecord(cn.ev[2 * ss], st));
    }
    const unsigned blocks = (unsigned)(((1LL << nout) + 255) / 256);
    if (cn.elem == 8) tnk::root_slice_sum<float2><<<blocks, 256, 0, st>>>(p, nfree, nout, out);
    else tnk::root_slice_sum<double2><<<blocks, 256, 0, st>>>(p, nfree, nout, out);
    CK(cudaGetLastError());
    if (cn.trace) {
        CK(cudaEventRecord(cn.ev[2 * ss + 1], st));
        cn.ev_pending[ss] = 1;
        cn.tr_kernel[ss] = 3;
    }
    return TN_OK;
}

// One execution of a compiled network: batch gathers, steps, FP64 slice sum into out.
int execute(CNet &cn, const uint64_t *d_closed, bool skip_beta_free, double2 *out, cudaStream_t st) {
    const long long fused = fused_root_step(cn);
    for (const Step &s : cn.steps) {
        if (skip_beta_free && !cn.tree.nodes[s.c].beta) continue;
        const size_t si = &s - cn.steps.data();
        if ((long long)si == fused) {
            // its operands' gathers still run here unless the row kernel reads them in place
            cn.cur_closed = d_closed;
            if (!(d_closed && row_fuses(cn, si))) RC(launch_gathers(cn, si, d_closed, st));
            continue;
        }
        if (cn.trace) {
            if (cn.ev_pending[si]) {  // fold the previous measurement in before reusing the events
                float ms = 0;
                CK(cudaEventSynchronize(cn.ev[2 * si + 1]));
                CK(cudaEventElapsedTime(&ms, cn.ev[2 * si], cn.ev[2 * si + 1]));
                cn.tr_ms[si] += ms;
                cn.tr_launches[si]++;
                cn.ev_pending[si] = 0;
            }
            CK(cudaEventRecord(cn.ev[2 * si], st));
        }
        cn.cur_closed = d_closed;
        const int var = si < cn.variant.size() && cn.variant[si] >= 0 ? cn.variant[si] : default_variant(cn, si);
        const bool in_place = d_closed && reads_in_place(cn, si, var);
        if (!in_place) RC(launch_gathers(cn, si, d_closed, st));
        if (cn.elem == 8) RC(launch_step<float2>(cn, s, st));
        else RC(launch_step<double2>(cn, s, st));
        if (cn.calibrating) {
            const long long n = 1LL << cn.tree.nodes[s.c].layout.size();
            for (long long v = 0; v < cn.cp.nver[s.c]; v++) {
                const char *base = static_cast<const char *>(cn.arena.p) + cn.cp.off[s.c] + v * n * 8;
                tnk::absmax_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 1024), 256, 0, st>>>(
                    base, n, cn.fmt[s.c], static_cast<int *>(cn.absmax.p) + s.c);
            }
            CK(cudaGetLastError());
        }
        if (cn.trace) {
            CK(cudaEventRecord(cn.ev[2 * si + 1], st));
            cn.ev_pending[si] = 1;
        }
    }
    if (fused >= 0) {
        cn.cur_closed = d_closed;
        return launch_root_slice_sum(cn, (size_t)fused, out, st);
    }
    return launch_slice_sum(cn, out, st);
}

// Kernel autotuning: the variant chosen for a step shape (precision and formats, fold,
// bit counts, versions) is cached for the process and shared by every plan.
std::mutex g_tune_mu;
std::map<std::vector<long long>, int> g_tune;

std::vector<long long> tune_key(const CNet &cn, size_t si) {
    const Step &s = cn.steps[si];
    const bool ipa = cn.cp.tc_inplace.size() > si && cn.cp.tc_inplace[si][0];
    const bool ipb = cn.cp.tc_inplace.size() > si && cn.cp.tc_inplace[si][1];
    return {cn.elem, cn.use_tc.empty() ? 0 : cn.use_tc[si], cn.cp.fold.empty() ? 0 : cn.cp.fold[si], cn.fmt[s.a],
            cn.fmt[s.c], s.nbat, s.nm, s.nn, s.nk, cn.cp.nver[s.c], ipa + 2 * ipb + 4 * stack_fits(cn, si, 128)};
}

// Fill in every step's variant that is known (single candidate, autotuning off, or a
// cached choice); true if some step still has to be timed.
bool resolve_variants(CNet &cn) {
    cn.variant.resize(cn.steps.size(), -1);
    bool need = false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (size_t si = 0; si < cn.steps.size(); si++) {
        if (cn.variant[si] >= 0) continue;
        const std::vector<int> c = step_variants(cn, si);
        if (cn.autotune >= 2 && !c.empty()) {
            cn.variant[si] = c[(si + (size_t)(cn.autotune - 2)) % c.size()];
            continue;
        }
        // steps under ~50 us (estimated) keep the shape rules: timing them costs more
        // than any choice can gain
        const double work = cn.steps[si].flops_per_version * (double)cn.cp.nver[cn.steps[si].c];
        if (cn.autotune <= 0 || c.size() <= 1 || work < 1e9) {
            cn.variant[si] = c.size() == 1 ? c[0] : default_variant(cn, si);
            continue;
        }
        auto it = g_tune.find(tune_key(cn, si));
        if (it != g_tune.end()) cn.variant[si] = it->second;
        else need = true;
    }
    return need;
}

// One full execution that times each applicable variant of every step still unchosen
// (one warm-up launch, then two timed launches, CUDA events on the plan's stream),
// keeps the fastest and then runs it, so `out` is written as by execute().
template <typename T>
int tune_execute(CNet &cn, const uint64_t *d_closed, double2 *out, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        tn_set_error("cudaEventCreate failed");
        return TN_EDEVICE;
    }
    int rc = TN_OK;
    cn.cur_closed = d_closed;
    for (size_t si = 0; si < cn.steps.size() && rc == TN_OK; si++) {
        const Step &s = cn.steps[si];
        rc = launch_gathers(cn, si, d_closed, st);
        if (rc == TN_OK && cn.variant[si] < 0) {
            int best = -1;
            float best_ms = 0;
            for (int v : step_variants(cn, si)) {
                rc = launch_variant<T>(cn, s, st, v);
                if (rc == TN_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = TN_EDEVICE;
                for (int r = 0; r < 2 && rc == TN_OK; r++) rc = launch_variant<T>(cn, s, st, v);
                float ms = 0;
                if (rc == TN_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)) {
                    tn_set_error("autotune: event timing failed");
                    rc = TN_EDEVICE;
                }
                if (rc != TN_OK) break;
                if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
            }
            if (rc == TN_OK) {
                cn.variant[si] = best;
                std::lock_guard<std::mutex> lock(g_tune_mu);
                g_tune[tune_key(cn, si)] = best;
            }
        }
        if (rc == TN_OK) rc = launch_step<T>(cn, s, st);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RC(rc);
    return launch_slice_sum(cn, out, st);
}

// fp16 split: the first execution runs with bf16 split operands and records every
// node's largest |re|, |im|; each fp16-stored tensor then gets the power-of-two scale
// putting that maximum at 2^8 (FP16 keeps values down to 2^-22 of it normal).
int calibrate_fp16(DevMem &mem, CNet &cn, const uint64_t *d_closed, double2 *out, cudaStream_t st, double budget) {
    const int NN = (int)cn.tree.nodes.size();
    RC(ensure(mem, cn.absmax, NN * sizeof(int)));
    CK(cudaMemsetAsync(cn.absmax.p, 0, NN * sizeof(int), st));
    cn.calibrating = true;
    int rc = execute(cn, d_closed, false, out, st);
    cn.calibrating = false;
    RC(rc);
    std::vector<int> bits(NN);
    CK(cudaMemcpyAsync(bits.data(), cn.absmax.p, NN * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cn.scale.assign(NN, 1.0f);
    for (int x = 0; x < NN; x++) {
        double mx = 0;
        if (cn.tree.nodes[x].ch[0] < 0) {
            for (const cplx &v : cn.net.leaves[x].data) mx = std::max(mx, std::max(std::fabs(v.real()), std::fabs(v.imag())));
        } else {
            float f;
            std::memcpy(&f, &bits[x], sizeof(f));
            mx = f;
        }
        if (mx > 0 && std::isfinite(mx)) cn.scale[x] = (float)std::ldexp(1.0, 8 - (int)std::ceil(std::log2(mx)));
    }
    cn.calibrated = true;
    cn.prec_active = TN_PREC_FP16X2;
    std::vector<uint64_t> slices = cn.cp.slices;
    drop_graphs(cn);
    assign_formats(cn);
    RC(setup_leaves(mem, cn));
    return prepare_call(mem, cn, slices, budget);
}

cudaStream_t capture_stream() {
    static thread_local cudaStream_t s = nullptr;
    if (!s) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    return s;
}

// execute() through a CUDA graph: the first execution for a (call plan, buffers, stem
// mode) is captured on an internal stream, later ones replay the graph on `st`.
int execute_graphed(DevMem &mem, CNet &cn, const uint64_t *d_closed, bool skip_beta_free, double2 *out,
                    cudaStream_t st, double budget) {
    if (cn.prec == TN_PREC_FP16X2 && !cn.calibrated) {
        RC(calibrate_fp16(mem, cn, d_closed, out, st, budget));
        skip_beta_free = false;  // the stem was recomputed in the calibration formats
    }
    if (resolve_variants(cn)) {
        drop_graphs(cn);
        return cn.elem == 8 ? tune_execute<float2>(cn, d_closed, out, st) : tune_execute<double2>(cn, d_closed, out, st);
    }
    static const bool disabled = getenv("TN_NO_GRAPH") != nullptr;
    if (cn.trace || disabled) return execute(cn, d_closed, skip_beta_free, out, st);
    const int gi = skip_beta_free ? 1 : 0;
    if (cn.graph[gi] && (cn.graph_key[gi][0] != d_closed || cn.graph_key[gi][1] != out)) {
        cudaGraphExecDestroy(cn.graph[gi]);
        cn.graph[gi] = nullptr;
    }
    if (!cn.graph[gi]) {
        cudaStream_t cs = capture_stream();
        if (!cs) return execute(cn, d_closed, skip_beta_free, out, st);
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int rc = execute(cn, d_closed, skip_beta_free, out, cs);
        cudaGraph_t g = nullptr;
        cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess || !g) {
            tn_set_error(std::string("graph capture failed: ") + cudaGetErrorString(ec));
            return TN_EDEVICE;
        }
        cudaError_t ei = cudaGraphInstantiate(&cn.graph[gi], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            cn.graph[gi] = nullptr;
            tn_set_error(std::string("graph instantiation failed: ") + cudaGetErrorString(ei));
            return TN_EDEVICE;
        }
        cn.graph_key[gi][0] = d_closed;
        cn.graph_key[gi][1] = out;
    }
    CK(cudaGraphLaunch(cn.graph[gi], st));
    return TN_OK;
}

// Compile (and re-materialise the leaves) for explicit-version legs E, if not current.
int ensure_variant(DevMem &mem, CNet &cn, uint64_t E) {
    if (cn.compiled && cn.E == E) return TN_OK;
    drop_graphs(cn);
    RC(tn_compile(cn.net, cn.tree, E, cn.steps, cn.elem == 8 && cn.prec != TN_PREC_C64));
    cn.E = E;
    cn.compiled = true;
    cn.cp.valid = false;
    assign_formats(cn);
    return setup_leaves(mem, cn);
}


// After a synchronising call: a bounded device wait that gave up is reported once.
int check_err(CNet &cn, cudaStream_t st) {
    if (!cn.d_err) return TN_OK;
    int h = 0;
    CK(cudaMemcpyAsync(&h, cn.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h) {
        CK(cudaMemsetAsync(cn.d_err, 0, sizeof(int), st));
        tn_set_error("a bounded device-side wait gave up (tensor-core step)");
        return TN_ETIMEOUT;
    }
    return TN_OK;
}

int build_cnet(const Merged &mg, CNet &cn, const tn_plan_opts &o, const int32_t *order, int n_order,
               DevMem &mem, int elem) {
    (void)mg;
    cn.elem = elem;
    uint64_t E0 = 0;
    tn_cost_settings(cn.net, o);
    if (elem != 8 || cn.prec == TN_PREC_C64) cn.net.tc_flop_rate = 0;
    RC(tn_tree_and_compile(cn.net, o, order, n_order, nullptr, cn.tree, cn.steps, &E0,
                           elem == 8 && cn.prec != TN_PREC_C64));
    cn.E = E0;
    cn.compiled = true;
    assign_formats(cn);
    return setup_leaves(mem, cn);
}

}  // namespace

// ---------------------------------------------------------------- sampling jobs

namespace {

// Device bytes of one execution on slice set sl (arena, leaves, per-group buffers, slack)
// and its algorithmic FLOPs for the first and each later batch group; host only.
int estimate_call(tn_plan_s *p, const std::vector<uint64_t> &sl, int64_t *bytes, double *flops_first,
                  double *flops_next) {
    const uint64_t E = explicit_legs(sl, (int)p->I.size());
    Tree t = p->amp.tree;
    std::vector<Step> steps;
    RC(tn_compile(p->amp.net, t, E, steps, p->amp.prec != TN_PREC_C64));
    CallLayout lay;
    layout_call(t, steps, E, 8, sl, lay);
    const long long T = 1LL << p->log2T;
    if (bytes) *bytes = (int64_t)(lay.arena_bytes + 2 * p->amp.leaf_bytes + T * (64 * 16 + 64)) + (64ll << 20);
    if (flops_first) *flops_first = lay.flops;
    if (flops_next) *flops_next = lay.flops_beta;
    return TN_OK;
}

// Batches a job draws for N samples at acceptance about 1/alpha: 10% above the mean
// need, plus 8 standard deviations and 64, rounded up to whole groups of T.
int64_t job_groups_for(int64_t N, double alpha, long long T) {
    const double need = 1.1 * alpha * (double)N + 8.0 * std::sqrt(alpha * (double)N) + 64.0;
    return std::max<int64_t>(1, (int64_t)std::ceil(need / (double)T));
}

}  // namespace

struct tn_job_s {
    tn_plan_s *p = nullptr;
    std::vector<uint64_t> slices;
    double F = 1.0, alpha = 2.0;
    int64_t N = 0, chunk = 1, n_chunks = 0, groups = 0;
    uint64_t seed = 0;
    std::vector<char> done;
    int64_t chunks_done = 0;
    double flops_done = 0, flops_chunk = 0;
    DBuf d_jall, d_acc;              // batch patterns and summed amplitudes of every batch
    DBuf d_accept, d_bits, d_eps, d_pick;
};

namespace {

// Reorder a selection X x {0,1}^free (tn_select's order: partial assignments, then the
// free legs' values) so that the free legs that add the least work when they vary inside
// a chunk vary fastest.  Varying leg e inside a chunk doubles every tensor below which e
// is sliced (it becomes a layout bit), while the steps that do not depend on e run once for
// the whole chunk; batch steps count once per batch group.  Legs are taken greedily by the
// job's FLOPs per slice, up to 12 of them.
int order_chunk_legs(tn_plan_s *p, double f, double groups, std::vector<uint64_t> &slices) {
    const int nI = (int)p->I.size();
    if (nI == 0 || nI > 40) return TN_OK;
    uint64_t smask = 0;
    if (f < 1.0)
        for (int e : p->norm_S) smask |= 1ull << e;
    std::vector<int> freeb;
    for (int e = 0; e < nI; e++)
        if (!((smask >> e) & 1)) freeb.push_back(e);
    const size_t per = size_t(1) << freeb.size();
    if (freeb.empty() || slices.size() % per) return TN_OK;
    // per-slice FLOPs and slice dependences of every step (all sliced legs explicit)
    Tree t = p->amp.tree;
    std::vector<Step> steps;
    const uint64_t all = nI >= 64 ? ~0ull : ((1ull << nI) - 1);
    RC(tn_compile(p->amp.net, t, all, steps, p->amp.prec != TN_PREC_C64));
    std::vector<double> w(steps.size());
    std::vector<uint64_t> dep(steps.size());
    for (size_t i = 0; i < steps.size(); i++) {
        w[i] = steps[i].flops_per_version * (t.nodes[steps[i].c].beta ? groups : 1.0);
        dep[i] = t.nodes[steps[i].c].dep;
    }
    auto per_slice = [&](uint64_t V) {
        double c = 0;
        for (size_t i = 0; i < steps.size(); i++) c += w[i] * std::ldexp(1.0, __builtin_popcountll(dep[i] & V));
        return c / std::ldexp(1.0, __builtin_popcountll(V));
    };
    std::vector<int> V;
    uint64_t vm = 0;
    while (V.size() < std::min<size_t>(12, freeb.size())) {
        int best = -1;
        double bc = 0;
        for (int e : freeb) {
            if ((vm >> e) & 1) continue;
            const double c = per_slice(vm | (1ull << e));
            if (best < 0 || c < bc) { best = e; bc = c; }
        }
        V.push_back(best);
        vm |= 1ull << best;
    }
    std::vector<int> rest;
    for (int e : freeb)
        if (!((vm >> e) & 1)) rest.push_back(e);
    std::vector<uint64_t> out;
    out.reserve(slices.size());
    for (size_t i = 0; i < slices.size(); i += per) {
        const uint64_t base = slices[i];  // the block's member with every free leg at 0
        for (uint64_t r2 = 0; r2 < (1ull << rest.size()); r2++) {
            uint64_t s2 = base;
            for (size_t u = 0; u < rest.size(); u++) s2 |= ((r2 >> u) & 1ull) << rest[u];
            for (uint64_t r1 = 0; r1 < (1ull << V.size()); r1++) {
                uint64_t s1 = s2;
                for (size_t u = 0; u < V.size(); u++) s1 |= ((r1 >> u) & 1ull) << V[u];
                out.push_back(s1);
            }
        }
    }
    slices.swap(out);
    return TN_OK;
}

void job_fill_info(const tn_job_s *j, tn_job_info *info) {
    if (!info) return;
    info->n_slices = (int64_t)j->slices.size();
    info->F = j->F;
    info->chunk_slices = j->chunk;
    info->n_chunks = j->n_chunks;
    info->groups = j->groups;
    info->T = 1LL << j->p->log2T;
    info->chunks_done = j->chunks_done;
    info->flops_done = j->flops_done;
    info->flops_chunk = j->flops_chunk;
}

void job_release(tn_job_s *j) {
    DevMem &m = j->p->mem;
    for (DBuf *b : {&j->d_jall, &j->d_acc, &j->d_accept, &j->d_bits, &j->d_eps, &j->d_pick}) release(m, *b);
}

}  // namespace

// ---------------------------------------------------------------- C-ABI

extern "C" {

const char *tn_last_error(void) { return g_err.c_str(); }

const char *tn_strerror(int code) {
    switch (code) {
        case TN_OK: return "ok";
        case TN_EINVAL: return "invalid argument";
        case TN_ENOMEM: return "out of memory or HBM budget exceeded";
        case TN_ETIMEOUT: return "device wait timed out";
        case TN_EDEVICE: return "CUDA device error";
        case TN_EUNSUPPORTED: return "unsupported request";
        default: return "unknown error";
    }
}

void tn_plan_opts_default(tn_plan_opts *o) {
    std::memset(o, 0, sizeof(*o));
    o->precision = TN_PREC_C64;
    o->log2_batches = 8;
    o->order_seed = 0;
    o->order_trials = 64;
    o->n_auto_sliced = 0;
    o->hbm_budget_bytes = 64.0 * (1ull << 30);
    o->max_norm_flops = 2e15;
    o->autotune = 1;
    o->fuse_root_sum = 0;
    o->job_groups = 1;
}

int tn_circuit_load(const void *buf, size_t len, tn_circuit_h *out) {
    if (!out) { tn_set_error("null output handle"); return TN_EINVAL; }
    *out = nullptr;
    auto *c = new (std::nothrow) tn_circuit_s;
    if (!c) return TN_ENOMEM;
    int rc = tn_parse_circuit(buf, len, c);
    if (rc != TN_OK) { delete c; return rc; }
    *out = c;
    return TN_OK;
}

void tn_circuit_destroy(tn_circuit_h c) { delete c; }

int tn_plan(tn_circuit_h c, const int32_t *order, int32_t n_order, const tn_edge *sliced, int32_t n_sliced,
            const int32_t *open_qubits, int32_t n_open, const tn_plan_opts *opts, tn_plan_h *out) {
    if (!c || !out || (n_open > 0 && !open_qubits) || n_open < 0 || n_open > 16) {
        tn_set_error("tn_plan: bad arguments (need circuit, output handle, 0 <= n_open <= 16)");
        return TN_EINVAL;
    }
    *out = nullptr;
    tn_plan_opts o;
    if (opts) o = *opts;
    else tn_plan_opts_default(&o);
    if (o.log2_batches < 0 || o.log2_batches > 16) { tn_set_error("log2_batches must be in [0,16]"); return TN_EINVAL; }
    if (o.precision != TN_PREC_C64 && o.precision != TN_PREC_BF16X2 && o.precision != TN_PREC_FP16X2) {
        tn_set_error("tn_plan: unknown precision");
        return TN_EINVAL;
    }
    if (sliced && (n_sliced < 0 || n_sliced > 62)) { tn_set_error("n_sliced must be in [0,62]"); return TN_EINVAL; }
    if (!sliced && (o.n_auto_sliced < 0 || o.n_auto_sliced > 62)) { tn_set_error("n_auto_sliced in [0,62]"); return TN_EINVAL; }
    if (o.max_log2_tensor < 0 || o.max_log2_tensor > 40) { tn_set_error("max_log2_tensor in [0,40]"); return TN_EINVAL; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) { tn_set_error("no CUDA device"); return TN_EDEVICE; }
    auto *p = new (std::nothrow) tn_plan_s;
    if (!p) return TN_ENOMEM;
    p->circ = *c;
    p->opts = o;
    p->mem.alloc = o.alloc;
    p->mem.free = o.free;
    p->mem.ctx = o.alloc_ctx;
    p->mem.stream = static_cast<cudaStream_t>(o.stream);
    p->budget = o.hbm_budget_bytes > 0 ? o.hbm_budget_bytes : 64.0 * (1ull << 30);
    tn_merge(p->circ, p->mg);
    p->open.assign(open_qubits, open_qubits + n_open);
    p->log2T = o.log2_batches;
    auto fail = [&](int rc) {
        free_cnet(p->mem, p->amp);
        delete p;
        return rc;
    };
    uint64_t E0 = 0;
    int rc = tn_plan_build_host(p->mg, o, order, n_order, sliced, n_sliced, p->open, p->I, p->amp.net,
                                p->amp.tree, p->amp.steps, p->closed, &E0);
    if (rc) return fail(rc);
    if (p->closed.empty()) p->log2T = 0;
    p->amp.elem = 8;
    p->amp.E = E0;
    p->amp.compiled = true;
    p->amp.prec = o.precision;
    p->amp.autotune = o.autotune;
    p->amp.fuse_root = o.fuse_root_sum != 0;
    assign_formats(p->amp);
    rc = setup_leaves(p->mem, p->amp);
    if (rc) return fail(rc);
    *out = p;
    return TN_OK;
}

void tn_plan_destroy(tn_plan_h p) {
    if (!p) return;
    free_cnet(p->mem, p->amp);
    for (DBuf *b : {&p->d_closed, &p->d_amps, &p->d_j, &p->d_acc, &p->d_pick, &p->d_eps, &p->d_bits, &p->d_R, &p->d_X,
                    &p->d_xidx, &p->d_xamps, &p->d_xsum, &p->d_skey, &p->d_shist, &p->d_sgt, &p->d_seq, &p->d_sbits,
                    &p->d_sprob})
        release(p->mem, *b);
    cudaStreamSynchronize(p->mem.stream);
    delete p;
}

static void fill_info(const Merged &mg, const std::vector<int> &open, const std::vector<int> &closed, int log2T,
                      const std::vector<tn_edge> &I, const Network &net, const Tree &tree,
                      const std::vector<Step> &steps, tn_plan_info *info) {
    std::memset(info, 0, sizeof(*info));
    info->n_qubits = mg.n;
    info->n_open = (int)open.size();
    info->n_closed = (int)closed.size();
    info->log2_batches = closed.empty() ? 0 : log2T;
    info->n_leaves = (int)net.leaves.size();
    info->n_steps = (int)steps.size();
    info->n_sliced = (int)I.size();
    int mx = 0;
    double fl1 = 0;
    for (auto &nd : tree.nodes) mx = std::max(mx, nd.idx.count());
    for (auto &s : steps) fl1 += s.flops_per_version;
    info->log2_max_tensor = mx;
    info->flops_per_slice = fl1;
    info->flops_all_slices = tn_tree_cost(net, tree).flops;
}

int tn_plan_host(tn_circuit_h c, const int32_t *order, int32_t n_order, const tn_edge *sliced, int32_t n_sliced,
                 const int32_t *open_qubits, int32_t n_open, const tn_plan_opts *opts, tn_plan_info *info,
                 int32_t *steps_out, int32_t cap_steps, tn_edge *sliced_out, int32_t cap_sliced) {
    if (!c || !info || (n_open > 0 && !open_qubits) || n_open < 0 || n_open > 16) {
        tn_set_error("tn_plan_host: bad arguments");
        return TN_EINVAL;
    }
    tn_plan_opts o;
    if (opts) o = *opts;
    else tn_plan_opts_default(&o);
    Merged mg;
    tn_merge(*c, mg);
    std::vector<int> open(open_qubits, open_qubits + n_open), closed;
    std::vector<tn_edge> I;
    Network net;
    Tree tree;
    std::vector<Step> steps;
    RC(tn_plan_build_host(mg, o, order, n_order, sliced, n_sliced, open, I, net, tree, steps, closed, nullptr));
    fill_info(mg, open, closed, o.log2_batches, I, net, tree, steps, info);
    if (steps_out)
        for (int i = 0; i < (int)steps.size() && i < cap_steps; i++) {
            const Step &s = steps[i];
            int32_t *r = steps_out + 7 * i;
            r[0] = s.nbat; r[1] = s.nm; r[2] = s.nn; r[3] = s.nk;
            r[4] = __builtin_popcountll(tree.nodes[s.c].dep);
            r[5] = __builtin_popcountll(tree.nodes[s.a].dep);
            r[6] = __builtin_popcountll(tree.nodes[s.b].dep);
        }
    if (sliced_out)
        for (int i = 0; i < (int)I.size() && i < cap_sliced; i++) sliced_out[i] = I[i];
    return TN_OK;
}

int tn_sliced_vertex_select(tn_circuit_h c, const tn_edge *I, int32_t n_I, int32_t k, int32_t *s_index,
                            int32_t *k_out) {
    if (!c || (n_I > 0 && !I) || !k_out || k < 0) { tn_set_error("tn_sliced_vertex_select: bad arguments"); return TN_EINVAL; }
    Merged mg;
    tn_merge(*c, mg);
    std::vector<tn_edge> Iv(I, I + n_I);
    for (auto &e : Iv)
        if (e.qubit < 0 || e.qubit >= mg.n || e.segment < 0 || e.segment > mg.n2q[e.qubit]) {
            tn_set_error("tn_sliced_vertex_select: vertex out of range");
            return TN_EINVAL;
        }
    std::vector<int> S = tn_sliced_vertex_select(mg, Iv, k);
    *k_out = (int32_t)S.size();
    if (s_index)
        for (size_t t = 0; t < S.size(); t++) s_index[t] = S[t];
    return TN_OK;
}

int tn_plan_get_info(tn_plan_h p, tn_plan_info *info) {
    if (!p || !info) { tn_set_error("null argument"); return TN_EINVAL; }
    fill_info(p->mg, p->open, p->closed, p->log2T, p->I, p->amp.net, p->amp.tree, p->amp.steps, info);
    return TN_OK;
}

int tn_plan_sliced_edges(tn_plan_h p, tn_edge *out, int32_t cap, int32_t *n_out) {
    if (!p || !n_out) { tn_set_error("null argument"); return TN_EINVAL; }
    *n_out = (int32_t)p->I.size();
    if (out)
        for (int i = 0; i < (int)p->I.size() && i < cap; i++) out[i] = p->I[i];
    return TN_OK;
}

int tn_plan_estimate(tn_plan_h p, const uint64_t *slices, int64_t n_slices, int64_t *device_bytes,
                     double *flops_first, double *flops_next) {
    if (!p || !slices || n_slices <= 0) { tn_set_error("tn_plan_estimate: bad arguments"); return TN_EINVAL; }
    std::vector<uint64_t> sl(slices, slices + n_slices);
    const uint64_t E = explicit_legs(sl, (int)p->I.size());
    Tree t = p->amp.tree;
    std::vector<Step> steps;
    RC(tn_compile(p->amp.net, t, E, steps, p->amp.prec != TN_PREC_C64));
    CallLayout lay;
    layout_call(t, steps, E, 8, sl, lay);
    const long long T = 1LL << p->log2T;
    if (device_bytes)
        *device_bytes = (int64_t)(lay.arena_bytes + 2 * p->amp.leaf_bytes + T * (64 * 16 + 64)) + (64ll << 20);
    if (flops_first) *flops_first = lay.flops;
    if (flops_next) *flops_next = lay.flops_beta;
    return TN_OK;
}

int tn_contract(tn_plan_h p, const uint64_t *slices, int64_t n_slices, const uint64_t *closed_bits, int64_t n_batches,
                double *amps, int32_t flags) {
    if (!p || !slices || n_slices <= 0 || !amps || n_batches <= 0 || (!closed_bits && !p->closed.empty())) {
        tn_set_error("tn_contract: bad arguments");
        return TN_EINVAL;
    }
    const int nI = (int)p->I.size();
    std::vector<uint64_t> sl(slices, slices + n_slices);
    {
        std::vector<uint64_t> sorted = sl;
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) { tn_set_error("duplicate slice"); return TN_EINVAL; }
        if (nI < 64 && sorted.back() >> nI) { tn_set_error("slice sets bits beyond the sliced edges"); return TN_EINVAL; }
    }
    cudaStream_t st = p->mem.stream;
    RC(ensure_variant(p->mem, p->amp, explicit_legs(sl, nI)));
    RC(prepare_call(p->mem, p->amp, sl, p->budget));
    const long long T = 1LL << p->log2T;
    const int nopen = (int)p->open.size();
    const long long NA = 1LL << nopen;
    RC(ensure(p->mem, p->d_closed, T * sizeof(uint64_t)));
    RC(ensure(p->mem, p->d_amps, T * NA * sizeof(double2)));
    const bool dev = flags & TN_DEVICE_BUFFERS;
    for (long long g0 = 0; g0 < n_batches; g0 += T) {
        long long nb = std::min<long long>(T, n_batches - g0);
        CK(cudaMemsetAsync(p->d_closed.p, 0, T * sizeof(uint64_t), st));
        if (!p->closed.empty())
            CK(cudaMemcpyAsync(p->d_closed.p, closed_bits + g0, nb * sizeof(uint64_t),
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        RC(execute_graphed(p->mem, p->amp, static_cast<const uint64_t *>(p->d_closed.p), g0 > 0, static_cast<double2 *>(p->d_amps.p), st, p->budget));
        CK(cudaMemcpyAsync(amps + 2 * g0 * NA, p->d_amps.p, nb * NA * sizeof(double2),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    return check_err(p->amp, st);
}

int tn_xeb(tn_plan_h p, const uint64_t *slices, int64_t n_slices, const uint64_t *bitstrings, int64_t N, double *xeb,
           double *amps) {
    if (!p || !slices || n_slices <= 0 || !bitstrings || N <= 0 || !xeb) {
        tn_set_error("tn_xeb: bad arguments");
        return TN_EINVAL;
    }
    const int nI = (int)p->I.size();
    std::vector<uint64_t> sl(slices, slices + n_slices);
    {
        std::vector<uint64_t> sorted = sl;
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) { tn_set_error("duplicate slice"); return TN_EINVAL; }
        if (nI < 64 && sorted.back() >> nI) { tn_set_error("slice sets bits beyond the sliced edges"); return TN_EINVAL; }
    }
    const int n = p->mg.n;
    if (n < 64)
        for (int64_t t = 0; t < N; t++)
            if (bitstrings[t] >> n) { tn_set_error("tn_xeb: bitstring beyond the circuit's qubits"); return TN_EINVAL; }
    // each string's batch (its closed qubits, ascending) and entry (its open qubits in order)
    std::vector<uint64_t> cb((size_t)N, 0);
    std::vector<int32_t> idx((size_t)N, 0);
    for (int64_t t = 0; t < N; t++) {
        for (size_t c = 0; c < p->closed.size(); c++) cb[t] |= ((bitstrings[t] >> p->closed[c]) & 1ull) << c;
        for (size_t r = 0; r < p->open.size(); r++) idx[t] |= (int32_t)(((bitstrings[t] >> p->open[r]) & 1ull) << r);
    }
    cudaStream_t st = p->mem.stream;
    RC(ensure_variant(p->mem, p->amp, explicit_legs(sl, nI)));
    RC(prepare_call(p->mem, p->amp, sl, p->budget));
    const long long T = 1LL << p->log2T;
    const int nopen = (int)p->open.size();
    RC(ensure(p->mem, p->d_closed, T * sizeof(uint64_t)));
    RC(ensure(p->mem, p->d_amps, (T << nopen) * sizeof(double2)));
    RC(ensure(p->mem, p->d_xidx, T * sizeof(int32_t)));
    RC(ensure(p->mem, p->d_xamps, N * sizeof(double2)));
    RC(ensure(p->mem, p->d_xsum, (tnk::kNormGrid + 1) * sizeof(double)));
    double2 *xa = static_cast<double2 *>(p->d_xamps.p);
    for (long long g0 = 0; g0 < N; g0 += T) {
        const long long nb = std::min<long long>(T, N - g0);
        CK(cudaMemsetAsync(p->d_closed.p, 0, T * sizeof(uint64_t), st));
        if (!p->closed.empty())
            CK(cudaMemcpyAsync(p->d_closed.p, cb.data() + g0, nb * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(p->d_xidx.p, idx.data() + g0, nb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        RC(execute_graphed(p->mem, p->amp, static_cast<const uint64_t *>(p->d_closed.p), g0 > 0,
                           static_cast<double2 *>(p->d_amps.p), st, p->budget));
        tnk::pick_amplitudes<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
            static_cast<const double2 *>(p->d_amps.p), nopen, static_cast<const int32_t *>(p->d_xidx.p), nb, xa + g0);
        CK(cudaGetLastError());
    }
    double *part = static_cast<double *>(p->d_xsum.p);
    tnk::sum_norms<<<tnk::kNormGrid, 256, 0, st>>>(xa, N, part);
    tnk::norm_total<<<1, tnk::kNormGrid, 0, st>>>(part, part + tnk::kNormGrid);
    CK(cudaGetLastError());
    double sum = 0.0;
    CK(cudaMemcpyAsync(&sum, part + tnk::kNormGrid, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (amps) CK(cudaMemcpyAsync(amps, xa, N * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    RC(check_err(p->amp, st));
    *xeb = std::ldexp(sum, n) / (double)N - 1.0;
    return TN_OK;
}

int tn_spoof(tn_plan_h p, const uint64_t *slices, int64_t n_slices, uint64_t closed_pattern, int64_t N,
             uint64_t *bitstrings, double *probs) {
    const int nopen = p ? (int)p->open.size() : 0;
    if (!p || !slices || n_slices <= 0 || !bitstrings || N < 1 || nopen > 30 || N > (1LL << nopen) ||
        (p->closed.size() < 64 && (closed_pattern >> p->closed.size()))) {
        tn_set_error("tn_spoof: bad arguments");
        return TN_EINVAL;
    }
    const int nI = (int)p->I.size();
    std::vector<uint64_t> sl(slices, slices + n_slices);
    {
        std::vector<uint64_t> sorted = sl;
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) { tn_set_error("duplicate slice"); return TN_EINVAL; }
        if (nI < 64 && sorted.back() >> nI) { tn_set_error("slice sets bits beyond the sliced edges"); return TN_EINVAL; }
    }
    cudaStream_t st = p->mem.stream;
    RC(ensure_variant(p->mem, p->amp, explicit_legs(sl, nI)));
    RC(prepare_call(p->mem, p->amp, sl, p->budget));
    const long long T = 1LL << p->log2T, M = 1LL << nopen;
    RC(ensure(p->mem, p->d_closed, T * sizeof(uint64_t)));
    RC(ensure(p->mem, p->d_amps, (T << nopen) * sizeof(double2)));
    // the batch is batch 0 of one group (the group's other batches take pattern 0)
    CK(cudaMemsetAsync(p->d_closed.p, 0, T * sizeof(uint64_t), st));
    CK(cudaMemcpyAsync(p->d_closed.p, &closed_pattern, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    RC(execute_graphed(p->mem, p->amp, static_cast<const uint64_t *>(p->d_closed.p), false,
                       static_cast<double2 *>(p->d_amps.p), st, p->budget));
    const long long nblk = (M + tnk::kSelBlock - 1) / tnk::kSelBlock;
    RC(ensure(p->mem, p->d_skey, M * sizeof(unsigned long long)));
    RC(ensure(p->mem, p->d_shist, 256 * sizeof(unsigned int)));
    RC(ensure(p->mem, p->d_sgt, nblk * sizeof(unsigned int)));
    RC(ensure(p->mem, p->d_seq, nblk * sizeof(unsigned int)));
    RC(ensure(p->mem, p->d_sbits, N * sizeof(unsigned long long)));
    if (probs) RC(ensure(p->mem, p->d_sprob, N * sizeof(double)));
    auto *key = static_cast<unsigned long long *>(p->d_skey.p);
    auto *hist = static_cast<unsigned int *>(p->d_shist.p);
    const unsigned grid = (unsigned)std::min<long long>((M + 255) / 256, 8LL * num_sms());
    tnk::spoof_keys<<<grid, 256, 0, st>>>(static_cast<const double2 *>(p->d_amps.p), M, key);
    CK(cudaGetLastError());
    // radix select, most significant digit first: the N-th largest key, and how many of
    // the keys equal to it the selection takes
    unsigned long long prefix = 0, mask = 0;
    long long need = N;
    for (int shift = 56; shift >= 0; shift -= 8) {
        CK(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st));
        tnk::digit_hist<<<grid, 256, 0, st>>>(key, M, mask, prefix, shift, hist);
        CK(cudaGetLastError());
        unsigned int h[256];
        CK(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        int d = 255;
        long long above = 0;
        while (d > 0 && above + (long long)h[d] < need) above += h[d--];
        need -= above;
        prefix |= (unsigned long long)d << shift;
        mask |= 255ull << shift;
    }
    auto *gt = static_cast<unsigned int *>(p->d_sgt.p);
    auto *eq = static_cast<unsigned int *>(p->d_seq.p);
    tnk::sel_counts<<<(unsigned)nblk, tnk::kSelBlock, 0, st>>>(key, M, prefix, gt, eq);
    tnk::sel_scan<<<1, tnk::kSelBlock, 0, st>>>(gt, eq, (int)nblk);
    unsigned long long base = 0;
    for (size_t c = 0; c < p->closed.size(); c++) base |= ((closed_pattern >> c) & 1ull) << p->closed[c];
    tnk::OpenQubits oq;
    std::memset(&oq, 0, sizeof(oq));
    oq.n = nopen;
    for (int r = 0; r < nopen; r++) oq.q[r] = (int8_t)p->open[r];
    tnk::sel_write<<<(unsigned)nblk, tnk::kSelBlock, 0, st>>>(key, M, prefix, need, gt, eq, base, oq,
                                                               static_cast<unsigned long long *>(p->d_sbits.p),
                                                               probs ? static_cast<double *>(p->d_sprob.p) : nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(bitstrings, p->d_sbits.p, N * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    if (probs) CK(cudaMemcpyAsync(probs, p->d_sprob.p, N * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return check_err(p->amp, st);
}

int tn_partial_norms(tn_plan_h p, double f, int32_t *s_index, int32_t *k_out, double *R, int64_t cap_R) {
    if (!p || !(f > 0.0 && f <= 1.0) || !k_out) { tn_set_error("tn_partial_norms: bad arguments"); return TN_EINVAL; }
    const int k0 = (int)std::ceil(3.0 - std::log2(f));
    std::vector<int> spos = tn_sliced_vertex_select(p->mg, p->I, k0);
    const int k = (int)spos.size();
    *k_out = k;
    if (s_index)
        for (int t = 0; t < k; t++) s_index[t] = spos[t];
    if (R && cap_R < (int64_t(1) << k)) { tn_set_error("R capacity below 2^k"); return TN_EINVAL; }
    if (k > 20) { tn_set_error("k above 20"); return TN_EUNSUPPORTED; }
    std::vector<double> Rh(size_t(1) << k, 0.0);
    if (k == 0) Rh[0] = 1.0;
    else {
        std::vector<tn_edge> S;
        for (int e : spos) S.push_back(p->I[e]);
        // R in the plan's contraction precision (complex64 FFMA or split tensor cores);
        // the FP64 work is the reduction of the slice cut
        CNet cn;
        cn.prec = p->amp.prec;
        int rc = tn_build_norm_network(p->mg, S, cn.net);
        if (rc) return rc;
        {
            Tree t;
            TreeCost tc;
            tn_greedy_tree(cn.net, p->opts.order_seed, p->opts.order_trials > 0 ? p->opts.order_trials : 64, t, tc);
            const double cap = p->opts.max_norm_flops > 0 ? p->opts.max_norm_flops : 2e15;
            if (tc.flops > cap) {
                tn_set_error("tn_partial_norms: the norm network needs " + std::to_string(tc.flops) +
                             " FLOPs (limit " + std::to_string(cap) + ")");
                return TN_EUNSUPPORTED;
            }
        }
        rc = build_cnet(p->mg, cn, p->opts, nullptr, 0, p->mem, 8);
        if (rc) { free_cnet(p->mem, cn); return rc; }
        rc = prepare_call(p->mem, cn, {0ull}, p->budget);
        if (rc) { free_cnet(p->mem, cn); return rc; }
        DBuf out;
        rc = ensure(p->mem, out, (size_t(1) << k) * sizeof(double2));
        if (!rc) rc = execute(cn, nullptr, false, static_cast<double2 *>(out.p), p->mem.stream);
        std::vector<double2> tmp(size_t(1) << k);
        if (!rc && cudaMemcpyAsync(tmp.data(), out.p, tmp.size() * sizeof(double2), cudaMemcpyDeviceToHost,
                                   p->mem.stream) != cudaSuccess) rc = TN_EDEVICE;
        if (!rc && cudaStreamSynchronize(p->mem.stream) != cudaSuccess) rc = TN_EDEVICE;
        release(p->mem, out);
        free_cnet(p->mem, cn);
        cudaStreamSynchronize(p->mem.stream);
        if (rc) { if (rc == TN_EDEVICE) tn_set_error("norm network execution failed"); return rc; }
        for (size_t i = 0; i < tmp.size(); i++) Rh[i] = tmp[i].x;
    }
    if (R) std::copy(Rh.begin(), Rh.end(), R);
    p->norm_f = f;
    p->norm_S = spos;
    p->norm_R = Rh;
    return TN_OK;
}

int tn_slice_cut(const double *R, int32_t k, double f, void *stream, int32_t *X, int32_t *n_x, double *F) {
    if (!R || !X || !n_x || !F || k < 0 || k > 12) { tn_set_error("tn_slice_cut: bad arguments (k <= 12)"); return TN_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = 1 << k;
    void *buf[4] = {nullptr, nullptr, nullptr, nullptr};
    const size_t sz[4] = {n * sizeof(double), n * sizeof(int32_t), sizeof(int32_t), sizeof(double)};
    // every buffer taken is returned to the stream's pool on every exit path
    auto run = [&]() -> int {
        for (int i = 0; i < 4; i++) CK(cudaMallocAsync(&buf[i], sz[i], st));
        double *dR = static_cast<double *>(buf[0]);
        int32_t *dX = static_cast<int32_t *>(buf[1]), *dn = static_cast<int32_t *>(buf[2]);
        double *dF = static_cast<double *>(buf[3]);
        CK(cudaMemcpyAsync(dR, R, n * sizeof(double), cudaMemcpyHostToDevice, st));
        size_t smem = (size_t)n * (sizeof(double) + sizeof(int));
        tnk::slice_cut<<<1, 256, smem, st>>>(dR, k, f, dX, dn, dF);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(n_x, dn, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(F, dF, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        CK(cudaMemcpyAsync(X, dX, (size_t)(*n_x) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        return TN_OK;
    };
    int rc = run();
    for (int i = 0; i < 4; i++)
        if (buf[i] && cudaFreeAsync(buf[i], st) != cudaSuccess && rc == TN_OK) {
            tn_set_error("tn_slice_cut: cudaFreeAsync failed");
            rc = TN_EDEVICE;
        }
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == TN_OK) {
        tn_set_error("tn_slice_cut: stream synchronisation failed");
        rc = TN_EDEVICE;
    }
    return rc;
}

int tn_select(tn_plan_h p, double f, uint64_t *slices, int64_t cap, int64_t *n_slices, double *F) {
    if (!p || !n_slices || !F || !(f > 0.0)) { tn_set_error("tn_select: bad arguments"); return TN_EINVAL; }
    const int nI = (int)p->I.size();
    if (nI > 40) { tn_set_error("tn_select: more than 40 sliced edges"); return TN_EUNSUPPORTED; }
    std::vector<uint64_t> out;
    if (f >= 1.0) {
        *F = 1.0;
        for (uint64_t s = 0; s < (1ull << nI); s++) out.push_back(s);
    } else {
        int32_t k = 0;
        std::vector<int32_t> spos(64);
        std::vector<double> R;
        if (p->norm_f == f) { spos = p->norm_S; k = (int)spos.size(); R = p->norm_R; }
        else {
            int k0 = (int)std::ceil(3.0 - std::log2(f));
            R.resize(size_t(1) << std::min(k0, 20));
            RC(tn_partial_norms(p, f, spos.data(), &k, R.data(), (int64_t)R.size()));
            R.resize(size_t(1) << k);
            spos.resize(k);
        }
        std::vector<int32_t> X(size_t(1) << k);
        int32_t nx = 0;
        RC(tn_slice_cut(R.data(), k, f, p->mem.stream, X.data(), &nx, F));
        // X x {0,1}^{|I|-k}: free bits are the sliced edges outside S
        std::vector<int> freeb;
        for (int e = 0; e < nI; e++)
            if (std::find(spos.begin(), spos.end(), e) == spos.end()) freeb.push_back(e);
        for (int a = 0; a < nx; a++) {
            uint64_t base = 0;
            for (int t = 0; t < k; t++) base |= (uint64_t)((X[a] >> t) & 1) << spos[t];
            for (uint64_t r = 0; r < (1ull << freeb.size()); r++) {
                uint64_t s = base;
                for (size_t u = 0; u < freeb.size(); u++) s |= ((r >> u) & 1ull) << freeb[u];
                out.push_back(s);
            }
        }
    }
    *n_slices = (int64_t)out.size();
    if (slices) {
        if (cap < (int64_t)out.size()) { tn_set_error("tn_select: capacity below the slice-set size"); return TN_EINVAL; }
        std::copy(out.begin(), out.end(), slices);
    }
    return TN_OK;
}

int tn_draw_batches(uint64_t seed, uint64_t t0, int64_t T, int32_t b_bits, uint64_t *j, void *stream) {
    if (!j || T < 0 || b_bits < 0 || b_bits > 64) { tn_set_error("tn_draw_batches: bad arguments"); return TN_EINVAL; }
    if (T == 0) return TN_OK;
    tnk::draw_batches<<<(unsigned)((T + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(seed, t0, T, b_bits, j);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_rejection_sample(const double *p, int64_t T, int32_t b_bits, double alpha, uint64_t seed, uint64_t t0,
                        uint8_t *accept, int32_t *pick, void *stream) {
    if (!p || !accept || !pick || T < 0 || b_bits < 0 || b_bits > 58 || !(alpha > 0)) {
        tn_set_error("tn_rejection_sample: bad arguments");
        return TN_EINVAL;
    }
    if (T == 0) return TN_OK;
    tnk::SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.p = p;
    sp.T = T;
    sp.b_bits = b_bits;
    sp.alpha = alpha;
    sp.seed = seed;
    sp.t0 = t0;
    sp.accept = accept;
    sp.pick = pick;
    tnk::sampler<<<(unsigned)((T * 32 + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(sp);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return TN_OK;
}

int tn_plan_sync(tn_plan_h p) {
    if (!p) { tn_set_error("null plan"); return TN_EINVAL; }
    CK(cudaStreamSynchronize(p->mem.stream));
    return check_err(p->amp, p->mem.stream);
}

int tn_trace_enable(tn_plan_h p, int32_t on) {
    if (!p) { tn_set_error("null plan"); return TN_EINVAL; }
    CNet &cn = p->amp;
    const size_t ns = cn.steps.size();
    // one entry per step plus one for the FP64 slice sum
    if (on && cn.ev.size() != 2 * (ns + 1)) {
        for (auto &x : cn.ev) cudaEventDestroy(x);
        cn.ev.assign(2 * (ns + 1), nullptr);
        for (auto &x : cn.ev) CK(cudaEventCreate(&x));
    }
    cn.ev_pending.assign(ns + 1, 0);
    cn.tr_launches.assign(ns + 1, 0);
    cn.tr_ms.assign(ns + 1, 0.0);
    cn.tr_kernel.assign(ns + 1, -1);
    cn.trace = on != 0;
    return TN_OK;
}

int tn_trace_read(tn_plan_h p, tn_step_trace *out, int32_t cap, int32_t *n_out) {
    if (!p || !n_out) { tn_set_error("null argument"); return TN_EINVAL; }
    CNet &cn = p->amp;
    const int ns = (int)cn.steps.size();
    *n_out = ns;
    if (!cn.trace) return TN_OK;
    CK(cudaStreamSynchronize(p->mem.stream));
    for (int si = 0; si <= ns; si++)
        if (cn.ev_pending[si]) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, cn.ev[2 * si], cn.ev[2 * si + 1]));
            cn.tr_ms[si] += ms;
            cn.tr_launches[si]++;
            cn.ev_pending[si] = 0;
        }
    const auto &nodes = cn.tree.nodes;
    *n_out = ns + 1;
    if (ns < cap && out) {
        // the slice sum: 2 FP64 additions and one complex64 read per summed element
        tn_step_trace &t = out[ns];
        std::memset(&t, 0, sizeof(t));
        t.step = ns;
        t.launches = cn.tr_launches[ns];
        t.ms = cn.tr_ms[ns];
        const int root = cn.tree.root;
        const double nout = std::ldexp(1.0, (int)cn.net.out_layout.size());
        const double summed = (cn.cp.valid ? (double)cn.cp.root_nver : 1.0) *
                              std::ldexp(1.0, (int)nodes[root].layout.size() - (int)cn.net.out_layout.size());
        t.nver = cn.cp.valid ? cn.cp.root_nver : 1;
        t.flops_per_launch = 2.0 * nout * summed;
        t.bytes_per_launch = 8.0 * nout * summed + 16.0 * nout;
        t.kernel = cn.tr_kernel.size() > (size_t)ns && cn.tr_kernel[ns] == 3 ? 3 : 2;
    }
    for (int si = 0; si < ns && si < cap && out; si++) {
        const Step &s = cn.steps[si];
        tn_step_trace &t = out[si];
        std::memset(&t, 0, sizeof(t));
        t.step = si;
        t.launches = cn.tr_launches[si];
        t.ms = cn.tr_ms[si];
        long long nv = cn.cp.valid ? cn.cp.nver[s.c] : 1;
        t.nver = nv;
        t.flops_per_launch = s.flops_per_version * (double)nv;
        auto vbytes = [&](int x) {
            long long v = cn.cp.valid ? cn.cp.nver[x] : 1;
            int bits = (int)nodes[x].layout.size();
            return 8.0 * std::ldexp(1.0, bits) * (double)v;
        };
        t.bytes_per_launch = vbytes(s.a) + vbytes(s.b) + vbytes(s.c);
        t.nbat = s.nbat;
        t.nm = s.nm;
        t.nn = s.nn;
        t.nk = s.nk;
        t.kernel = cn.tr_kernel[si];
        // a gather launch precedes the step unless the row kernels read the operands in place
        const bool has = cn.cp.valid && cn.cp.gd_off[si + 1] > cn.cp.gd_off[si];
        const bool in_place = reads_in_place(cn, (size_t)si, t.kernel);
        t.gathers = has && !in_place ? 1 : 0;
        t.in_place = has && in_place ? 1 : 0;
    }
    return TN_OK;
}

int tn_sample_step(tn_plan_h p, const uint64_t *slices, int64_t n_slices, double F, uint64_t seed, uint64_t t0,
                   double alpha, int32_t reuse_stem, uint8_t *accept, uint64_t *bits, int32_t flags) {
    if (!p || !slices || n_slices <= 0 || !accept || !bits || !(alpha > 1.0) || !(F > 0.0)) {
        tn_set_error("tn_sample_step: bad arguments");
        return TN_EINVAL;
    }
    if (p->open.size() != 6) { tn_set_error("tn_sample_step: needs 6 open qubits"); return TN_EUNSUPPORTED; }
    std::vector<uint64_t> sl(slices, slices + n_slices);
    if (!(p->amp.cp.valid && p->amp.cp.slices == sl)) {
        RC(ensure_variant(p->mem, p->amp, explicit_legs(sl, (int)p->I.size())));
        RC(prepare_call(p->mem, p->amp, sl, p->budget));
    }
    cudaStream_t st = p->mem.stream;
    const long long T = 1LL << p->log2T;
    const int b_bits = (int)p->closed.size();
    RC(ensure(p->mem, p->d_j, T * sizeof(uint64_t)));
    RC(ensure(p->mem, p->d_amps, T * 64 * sizeof(double2)));
    RC(ensure(p->mem, p->d_pick, T * sizeof(int32_t)));
    const bool dev = flags & TN_DEVICE_BUFFERS;
    if (!dev) {
        RC(ensure(p->mem, p->d_acc, T));
        RC(ensure(p->mem, p->d_bits, T * sizeof(uint64_t)));
    }
    tnk::draw_batches<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(seed, t0, T, b_bits, static_cast<uint64_t *>(p->d_j.p));
    CK(cudaGetLastError());
    RC(execute_graphed(p->mem, p->amp, static_cast<const uint64_t *>(p->d_j.p), reuse_stem != 0, static_cast<double2 *>(p->d_amps.p), st, p->budget));
    tnk::SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.amps = static_cast<const double2 *>(p->d_amps.p);
    sp.invF_num = F;
    sp.T = T;
    sp.b_bits = b_bits;
    sp.alpha = alpha;
    sp.seed = seed;
    sp.t0 = t0;
    sp.accept = dev ? accept : static_cast<uint8_t *>(p->d_acc.p);
    sp.pick = static_cast<int32_t *>(p->d_pick.p);
    sp.j = static_cast<const uint64_t *>(p->d_j.p);
    sp.bits = dev ? bits : static_cast<uint64_t *>(p->d_bits.p);
    sp.n_open = 6;
    sp.n_closed = b_bits;
    for (int r = 0; r < 6; r++) sp.open_q[r] = (int8_t)p->open[r];
    for (int c = 0; c < b_bits; c++) sp.closed_q[c] = (int8_t)p->closed[c];
    tnk::sampler<<<(unsigned)((T * 32 + 255) / 256), 256, 0, st>>>(sp);
    CK(cudaGetLastError());
    if (!dev) {
        CK(cudaMemcpyAsync(accept, p->d_acc.p, T, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(bits, p->d_bits.p, T * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        RC(check_err(p->amp, st));
    }
    return TN_OK;
}

int tn_sample(tn_plan_h p, double f_target, int64_t N, uint64_t seed, double alpha, uint64_t *bitstrings,
              int32_t flags, tn_sample_stats *stats) {
    if (!p || N < 0 || !bitstrings || !(alpha > 1.0) || !(f_target > 0.0)) {
        tn_set_error("tn_sample: bad arguments (alpha > 1, f_target > 0)");
        return TN_EINVAL;
    }
    if (p->open.size() != 6) { tn_set_error("tn_sample: needs 6 open qubits (batches of 64)"); return TN_EUNSUPPORTED; }
    tn_sample_stats st_local;
    std::memset(&st_local, 0, sizeof(st_local));
    int64_t nsl = 0;
    double F = 1.0;
    RC(tn_select(p, f_target, nullptr, 0, &nsl, &F));
    std::vector<uint64_t> sl((size_t)nsl);
    RC(tn_select(p, f_target, sl.data(), nsl, &nsl, &F));
    st_local.F = F;
    st_local.n_slices = nsl;
    cudaStream_t st = p->mem.stream;
    if (!(p->amp.cp.valid && p->amp.cp.slices == sl)) {
        // a slice set beyond one execution's memory runs as a chunked sampling job
        int64_t need = 0;
        RC(estimate_call(p, sl, &need, nullptr, nullptr));
        if ((double)need > p->budget) {
            tn_job_h job = nullptr;
            RC(tn_job_create(p, f_target, N, seed, alpha, 0, &job, nullptr));
            std::vector<uint64_t> res((size_t)N);
            int rc = tn_job_run(job, 0, job->n_chunks);
            if (rc == TN_OK) rc = tn_job_finish(job, res.data(), 0, &st_local);
            tn_job_destroy(job);
            RC(rc);
            if (flags & TN_DEVICE_BUFFERS) {
                CK(cudaMemcpyAsync(bitstrings, res.data(), (size_t)N * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
                CK(cudaStreamSynchronize(st));
            } else {
                std::copy(res.begin(), res.end(), bitstrings);
            }
            if (stats) *stats = st_local;
            return TN_OK;
        }
        RC(ensure_variant(p->mem, p->amp, explicit_legs(sl, (int)p->I.size())));
        RC(prepare_call(p->mem, p->amp, sl, p->budget));
    }
    const long long T = 1LL << p->log2T;
    const int b_bits = (int)p->closed.size();
    RC(ensure(p->mem, p->d_j, T * sizeof(uint64_t)));
    RC(ensure(p->mem, p->d_amps, T * 64 * sizeof(double2)));
    RC(ensure(p->mem, p->d_acc, T));
    RC(ensure(p->mem, p->d_pick, T * sizeof(int32_t)));
    RC(ensure(p->mem, p->d_eps, T * sizeof(double)));
    RC(ensure(p->mem, p->d_bits, T * sizeof(uint64_t)));
    std::vector<uint8_t> h_acc(T);
    std::vector<uint64_t> h_bits(T);
    std::vector<double> h_eps(T);
    std::vector<uint64_t> result;
    result.reserve((size_t)N);
    const int64_t max_steps = (int64_t)std::ceil(8.0 * alpha * (double)N) + 4096;
    int64_t t = 0;
    double eps_sum = 0;
    int group = 0;
    tnk::SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.amps = static_cast<const double2 *>(p->d_amps.p);
    sp.invF_num = F;
    sp.T = T;
    sp.b_bits = b_bits;
    sp.alpha = alpha;
    sp.seed = seed;
    sp.accept = static_cast<uint8_t *>(p->d_acc.p);
    sp.pick = static_cast<int32_t *>(p->d_pick.p);
    sp.eps = static_cast<double *>(p->d_eps.p);
    sp.j = static_cast<const uint64_t *>(p->d_j.p);
    sp.bits = static_cast<uint64_t *>(p->d_bits.p);
    sp.n_open = 6;
    sp.n_closed = b_bits;
    for (int r = 0; r < 6; r++) sp.open_q[r] = (int8_t)p->open[r];
    for (int c = 0; c < b_bits; c++) sp.closed_q[c] = (int8_t)p->closed[c];
    while ((int64_t)result.size() < N && t < max_steps) {
        tnk::draw_batches<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(seed, (uint64_t)t, T, b_bits,
                                                                         static_cast<uint64_t *>(p->d_j.p));
        CK(cudaGetLastError());
        RC(execute_graphed(p->mem, p->amp, static_cast<const uint64_t *>(p->d_j.p), group > 0, static_cast<double2 *>(p->d_amps.p), st, p->budget));
        sp.t0 = (uint64_t)t;
        tnk::sampler<<<(unsigned)((T * 32 + 255) / 256), 256, 0, st>>>(sp);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h_acc.data(), p->d_acc.p, T, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_bits.data(), p->d_bits.p, T * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_eps.data(), p->d_eps.p, T * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const long long take = std::min<long long>(T, max_steps - t);
        for (long long i = 0; i < take; i++) {
            eps_sum += h_eps[i];
            if (h_acc[i]) {
                st_local.accepted++;
                if ((int64_t)result.size() < N) result.push_back(h_bits[i]);
            }
        }
        st_local.flops += group == 0 ? p->amp.cp.flops_all : p->amp.cp.flops_beta;
        t += take;
        group++;
    }
    st_local.steps = t;
    st_local.eps_hat = t > 0 ? eps_sum / (double)t : 0.0;
    if (flags & TN_DEVICE_BUFFERS) {
        CK(cudaMemcpyAsync(bitstrings, result.data(), result.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::copy(result.begin(), result.end(), bitstrings);
    }
    if (stats) *stats = st_local;
    RC(check_err(p->amp, st));
    if ((int64_t)result.size() < N) {
        tn_set_error("tn_sample: step limit reached before N accepted samples");
        return TN_EINVAL;
    }
    return TN_OK;
}

int tn_plan_test_stall(tn_plan_h p, int64_t cycles) {
    if (!p || cycles < 0 || cycles > 4000000000LL) { tn_set_error("tn_plan_test_stall: bad arguments"); return TN_EINVAL; }
    p->amp.tc_stall = cycles;
    drop_graphs(p->amp);  // the captured launches hold the previous setting
    return TN_OK;
}

int tn_job_create(tn_plan_h p, double f_target, int64_t N, uint64_t seed, double alpha, int64_t max_chunk_slices,
                  tn_job_h *out, tn_job_info *info) {
    if (!p || !out || N < 1 || !(alpha > 1.0) || !(f_target > 0.0) || max_chunk_slices < 0) {
        tn_set_error("tn_job_create: bad arguments (N >= 1, alpha > 1, f_target > 0)");
        return TN_EINVAL;
    }
    if (p->open.size() != 6) { tn_set_error("tn_job_create: needs 6 open qubits (batches of 64)"); return TN_EUNSUPPORTED; }
    *out = nullptr;
    std::unique_ptr<tn_job_s> j(new tn_job_s());
    j->p = p;
    j->N = N;
    j->seed = seed;
    j->alpha = alpha;
    int64_t nsl = 0;
    RC(tn_select(p, f_target, nullptr, 0, &nsl, &j->F));
    j->slices.resize((size_t)nsl);
    RC(tn_select(p, f_target, j->slices.data(), nsl, &nsl, &j->F));
    const long long T = 1LL << p->log2T;
    j->groups = job_groups_for(N, alpha, T);
    RC(order_chunk_legs(p, f_target, (double)j->groups, j->slices));
    const double job_bytes = (double)j->groups * (double)T * (64.0 * 16.0 + 8.0 + 1.0 + 8.0 + 8.0 + 4.0);
    // chunks: aligned runs of a power of two of consecutive slices of the selection
    // (the lowest free legs vary inside a chunk, so every chunk compiles alike)
    int64_t c = 1;
    while (c * 2 <= nsl && nsl % (c * 2) == 0 && (max_chunk_slices == 0 || c * 2 <= max_chunk_slices)) {
        int64_t b = 0;
        std::vector<uint64_t> sl(j->slices.begin(), j->slices.begin() + c * 2);
        RC(estimate_call(p, sl, &b, nullptr, nullptr));
        if ((double)b + job_bytes > 0.95 * p->budget) break;
        c *= 2;
    }
    {
        int64_t b = 0;
        std::vector<uint64_t> sl(j->slices.begin(), j->slices.begin() + c);
        RC(estimate_call(p, sl, &b, nullptr, nullptr));
        if ((double)b + job_bytes > p->budget) {
            tn_set_error("tn_job_create: one slice and the job's buffers exceed the HBM budget");
            return TN_ENOMEM;
        }
        double f1 = 0, f2 = 0;
        RC(estimate_call(p, sl, nullptr, &f1, &f2));
        j->flops_chunk = f1 + (double)(j->groups - 1) * f2;
    }
    j->chunk = c;
    j->n_chunks = nsl / c;
    j->done.assign((size_t)j->n_chunks, 0);
    DevMem &m = p->mem;
    const long long nb = j->groups * T;
    cudaStream_t st = m.stream;
    int rc = TN_OK;
    auto fail = [&](int r) { job_release(j.get()); return r; };
    if ((rc = ensure(m, j->d_jall, nb * sizeof(uint64_t))) || (rc = ensure(m, j->d_acc, nb * 64 * sizeof(double2))) ||
        (rc = ensure(m, j->d_accept, nb)) || (rc = ensure(m, j->d_bits, nb * sizeof(uint64_t))) ||
        (rc = ensure(m, j->d_eps, nb * sizeof(double))) || (rc = ensure(m, j->d_pick, nb * sizeof(int32_t))))
        return fail(rc);
    if (cudaMemsetAsync(j->d_acc.p, 0, nb * 64 * sizeof(double2), st) != cudaSuccess) {
        tn_set_error("tn_job_create: clearing the amplitude sums failed");
        return fail(TN_EDEVICE);
    }
    tnk::draw_batches<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(seed, 0, nb, (int)p->closed.size(),
                                                                    static_cast<uint64_t *>(j->d_jall.p));
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        tn_set_error("tn_job_create: batch draws failed");
        return fail(TN_EDEVICE);
    }
    job_fill_info(j.get(), info);
    *out = j.release();
    return TN_OK;
}

int tn_job_run(tn_job_h j, int64_t first, int64_t count) {
    if (!j || first < 0 || count < 0 || first + count > j->n_chunks) { tn_set_error("tn_job_run: bad chunk range"); return TN_EINVAL; }
    for (int64_t c = first; c < first + count; c++)
        if (j->done[(size_t)c]) { tn_set_error("tn_job_run: chunk " + std::to_string(c) + " already ran"); return TN_EINVAL; }
    tn_plan_s *p = j->p;
    cudaStream_t st = p->mem.stream;
    const long long T = 1LL << p->log2T;
    RC(ensure(p->mem, p->d_j, T * sizeof(uint64_t)));
    RC(ensure(p->mem, p->d_amps, T * 64 * sizeof(double2)));
    const uint64_t *jall = static_cast<const uint64_t *>(j->d_jall.p);
    double2 *acc = static_cast<double2 *>(j->d_acc.p);
    const unsigned agrid = (unsigned)std::min<long long>((T * 64 + 255) / 256, 8LL * num_sms());
    for (int64_t c = first; c < first + count; c++) {
        std::vector<uint64_t> sl(j->slices.begin() + c * j->chunk, j->slices.begin() + (c + 1) * j->chunk);
        RC(ensure_variant(p->mem, p->amp, explicit_legs(sl, (int)p->I.size())));
        RC(prepare_call(p->mem, p->amp, sl, p->budget));
        for (int64_t g = 0; g < j->groups; g++) {
            // the group's patterns go to the buffer the captured graphs read
            CK(cudaMemcpyAsync(p->d_j.p, jall + g * T, T * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
            RC(execute_graphed(p->mem, p->amp, static_cast<const uint64_t *>(p->d_j.p), g > 0,
                               static_cast<double2 *>(p->d_amps.p), st, p->budget));
            tnk::accumulate_amps<<<agrid, 256, 0, st>>>(acc + g * T * 64, static_cast<const double2 *>(p->d_amps.p),
                                                        T * 64);
            CK(cudaGetLastError());
        }
        j->flops_done += p->amp.cp.flops_all + (double)(j->groups - 1) * p->amp.cp.flops_beta;
        j->done[(size_t)c] = 1;
        j->chunks_done++;
    }
    CK(cudaStreamSynchronize(st));
    return check_err(p->amp, st);
}

int tn_job_get_info(tn_job_h j, tn_job_info *info) {
    if (!j || !info) { tn_set_error("tn_job_get_info: bad arguments"); return TN_EINVAL; }
    job_fill_info(j, info);
    return TN_OK;
}

int tn_job_amplitudes(tn_job_h j, int64_t g, double *amps) {
    if (!j || !amps || g < 0 || g >= j->groups) { tn_set_error("tn_job_amplitudes: bad arguments"); return TN_EINVAL; }
    const long long T = 1LL << j->p->log2T;
    cudaStream_t st = j->p->mem.stream;
    CK(cudaMemcpyAsync(amps, static_cast<const double2 *>(j->d_acc.p) + g * T * 64, T * 64 * sizeof(double2),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return TN_OK;
}

int tn_job_finish(tn_job_h j, uint64_t *bitstrings, int32_t flags, tn_sample_stats *stats) {
    if (!j || !bitstrings) { tn_set_error("tn_job_finish: bad arguments"); return TN_EINVAL; }
    if (j->chunks_done < j->n_chunks && !(flags & TN_JOB_PARTIAL)) {
        tn_set_error("tn_job_finish: " + std::to_string(j->n_chunks - j->chunks_done) + " chunks have not run");
        return TN_EINVAL;
    }
    tn_plan_s *p = j->p;
    cudaStream_t st = p->mem.stream;
    const long long T = 1LL << p->log2T, nb = j->groups * T;
    const int b_bits = (int)p->closed.size();
    tnk::SampleParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.amps = static_cast<const double2 *>(j->d_acc.p);
    sp.invF_num = j->F;
    sp.T = nb;
    sp.b_bits = b_bits;
    sp.alpha = j->alpha;
    sp.seed = j->seed;
    sp.t0 = 0;
    sp.accept = static_cast<uint8_t *>(j->d_accept.p);
    sp.pick = static_cast<int32_t *>(j->d_pick.p);
    sp.eps = static_cast<double *>(j->d_eps.p);
    sp.j = static_cast<const uint64_t *>(j->d_jall.p);
    sp.bits = static_cast<uint64_t *>(j->d_bits.p);
    sp.n_open = 6;
    sp.n_closed = b_bits;
    for (int r = 0; r < 6; r++) sp.open_q[r] = (int8_t)p->open[r];
    for (int c = 0; c < b_bits; c++) sp.closed_q[c] = (int8_t)p->closed[c];
    tnk::sampler<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(sp);
    CK(cudaGetLastError());
    std::vector<uint8_t> h_acc((size_t)nb);
    std::vector<uint64_t> h_bits((size_t)nb);
    std::vector<double> h_eps((size_t)nb);
    CK(cudaMemcpyAsync(h_acc.data(), j->d_accept.p, nb, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_bits.data(), j->d_bits.p, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_eps.data(), j->d_eps.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    tn_sample_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    int64_t got = 0;
    double eps_sum = 0;
    for (long long t = 0; t < nb; t++) {
        eps_sum += h_eps[(size_t)t];
        if (h_acc[(size_t)t]) {
            sst.accepted++;
            if (got < j->N) bitstrings[got++] = h_bits[(size_t)t];
        }
    }
    sst.F = j->F;
    sst.steps = nb;
    sst.eps_hat = eps_sum / (double)nb;
    sst.n_slices = (int64_t)j->slices.size();
    sst.flops = j->flops_done;
    if (stats) *stats = sst;
    if (got < j->N && !(flags & TN_JOB_PARTIAL)) {
        tn_set_error("tn_job_finish: " + std::to_string(got) + " of " + std::to_string(j->N) +
                     " samples accepted in the job's batches");
        return TN_EINVAL;
    }
    return TN_OK;
}

void tn_job_destroy(tn_job_h j) {
    if (!j) return;
    job_release(j);
    delete j;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free slice cut
//
// Some callers cannot allocate device memory from their call path: a process whose
// device memory is owned up front by another allocator (for example a serving loop
// that reserved all of HBM for plans and resident tensors), or code that must not
// enter the CUDA allocator at all (an allocation can wait on other work on the device
// and can fail when memory is fragmented).  tn_slice_cut_noalloc is tn_slice_cut for
// them: its scratch (the copy of R, the sorted indices, the count and the sum) lives in
// the static device array below, reserved when the library is loaded and held by every
// GPU that loads it until the process exits.

namespace {
constexpr int kCutMaxK = 12;                                               // 2^12 norms at most
constexpr size_t kCutRBytes = (size_t(1) << kCutMaxK) * sizeof(double);    // 32 KiB
constexpr size_t kCutXBytes = (size_t(1) << kCutMaxK) * sizeof(int32_t);   // 16 KiB
constexpr size_t kCutScratchBytes = kCutRBytes + kCutXBytes + 256;        // + count and sum
constexpr int kCutMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_cut_scratch[kCutScratchBytes];

namespace {
std::mutex g_cut_mu;
void *g_cut_dev_ptr[kCutMaxDevices] = {};

// Device address of g_cut_scratch on the current device.  Host code only has a
// host-side stand-in under that name, so the address is looked up once per device
// (with that device current) and cached.  The cache outlives a cudaDeviceReset, after
// which the module is reloaded at another address: callers that reset a device must
// not use this entry point afterwards in the same process.
int cut_scratch_address(void **out) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kCutMaxDevices) {
        tn_set_error("tn_slice_cut_noalloc: device ordinal outside the supported range");
        return TN_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_cut_mu);
    if (!g_cut_dev_ptr[dev]) {
        void *p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_cut_scratch));
        if (!p) {
            tn_set_error("tn_slice_cut_noalloc: no device address for the static scratch");
            return TN_EDEVICE;
        }
        g_cut_dev_ptr[dev] = p;
    }
    *out = g_cut_dev_ptr[dev];
    return TN_OK;
}
}  // namespace

extern "C" int tn_slice_cut_noalloc(const double *R, int32_t k, double f, void *stream, int32_t *X, int32_t *n_x,
                                    double *F) {
    if (!R || !X || !n_x || !F || k < 0) {
        tn_set_error("tn_slice_cut_noalloc: bad arguments");
        return TN_EINVAL;
    }
    if (k > kCutMaxK) {
        tn_set_error("tn_slice_cut_noalloc: k = " + std::to_string(k) + " exceeds the static scratch limit k <= " +
                     std::to_string(kCutMaxK));
        return TN_EINVAL;
    }
    void *base = nullptr;
    RC(cut_scratch_address(&base));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = 1 << k;
    unsigned char *b = static_cast<unsigned char *>(base);
    double *dR = reinterpret_cast<double *>(b);
    int32_t *dX = reinterpret_cast<int32_t *>(b + kCutRBytes);
    int32_t *dn = reinterpret_cast<int32_t *>(b + kCutRBytes + kCutXBytes);
    double *dF = reinterpret_cast<double *>(b + kCutRBytes + kCutXBytes + 128);
    // the array keeps the previous call's contents: clear the count and the sum
    CK(cudaMemsetAsync(b + kCutRBytes + kCutXBytes, 0, 256, st));
    CK(cudaMemcpyAsync(dR, R, n * sizeof(double), cudaMemcpyHostToDevice, st));
    size_t smem = (size_t)n * (sizeof(double) + sizeof(int));
    tnk::slice_cut<<<1, 256, smem, st>>>(dR, k, f, dX, dn, dF);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(n_x, dn, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(F, dF, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(X, dX, (size_t)(*n_x) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return TN_OK;
}
