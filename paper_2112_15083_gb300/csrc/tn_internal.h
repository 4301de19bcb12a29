// Internal structures of libtn: circuit, tensor network, contraction tree and the
// compiled step list.  Host-only declarations (shared by planner.cpp and engine.cu).
#pragma once

#include <algorithm>
#include <cstdint>
#include <complex>
#include <string>
#include <vector>

#include "tn.h"

using cplx = std::complex<double>;

// ------------------------------------------------------------------ errors
void tn_set_error(const std::string &msg);

// ------------------------------------------------------------------ circuit
struct TnGate {
    int arity;
    int q[2];
    cplx m[16];  // row-major (2^arity)^2
};

struct tn_circuit_s {
    int n = 0;
    std::vector<TnGate> gates;
};

int tn_parse_circuit(const void *buf, size_t len, tn_circuit_s *c);

// ------------------------------------------------------------------ index sets
constexpr int kMaxIdx = 1024;
struct Bits {
    uint64_t w[kMaxIdx / 64] = {};
    void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
    void clr(int i) { w[i >> 6] &= ~(1ull << (i & 63)); }
    bool has(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
    int count() const {
        int c = 0;
        for (auto x : w) c += __builtin_popcountll(x);
        return c;
    }
    Bits operator|(const Bits &o) const { Bits r; for (int i = 0; i < kMaxIdx / 64; i++) r.w[i] = w[i] | o.w[i]; return r; }
    Bits operator&(const Bits &o) const { Bits r; for (int i = 0; i < kMaxIdx / 64; i++) r.w[i] = w[i] & o.w[i]; return r; }
    Bits andnot(const Bits &o) const { Bits r; for (int i = 0; i < kMaxIdx / 64; i++) r.w[i] = w[i] & ~o.w[i]; return r; }
    bool any() const { for (auto x : w) if (x) return true; return false; }
    std::vector<int> list() const {
        std::vector<int> out;
        for (int i = 0; i < kMaxIdx / 64; i++) {
            uint64_t x = w[i];
            while (x) { int b = __builtin_ctzll(x); out.push_back(i * 64 + b); x &= x - 1; }
        }
        return out;
    }
};

// ------------------------------------------------------------------ network
// Leg kinds of a leaf tensor.
enum LegKind { LEG_NET = 0, LEG_SLICED = 1 };  // closed outputs are network legs (Network::closed_base)

struct Leaf {
    // data index = sum_t value(leg t) << t
    std::vector<int> kind;  // LegKind
    std::vector<int> ref;   // NET: network index id; SLICED: position e in I; CLOSED: closed pos c
    std::vector<cplx> data; // 2^legs
};

// A contraction network: leaves, index space, output indices.
struct Network {
    int n_idx = 0;                 // network index ids [0, n_idx)
    std::vector<Leaf> leaves;
    std::vector<int> out_layout;   // output index ids, LSB first
    int n_beta = 0;                // beta bits are network ids beta_base .. beta_base+n_beta-1
    int beta_base = -1;
    // Closed output legs are network ids closed_base .. closed_base+n_closed-1 (id of
    // closed position c = closed_base + c).  A tensor keeps them as ordinary legs (one
    // copy per value, shared by every batch) while it holds at most q_max of them; a
    // step whose result would hold more, or that meets a batch tensor, selects each
    // batch's values (a gather) and carries the beta bits instead.
    int closed_base = -1;
    int n_closed = 0;
    int q_max = 0;                 // -1: leaves with closed legs are in batch form from the start
    // Cost model: FLOP rate of tensor-core shaped steps (0: every step runs on FFMA), and
    // the largest operand + result footprint of one step (elements over all versions;
    // 0: unlimited) above which a tree is treated as infeasible.
    double tc_flop_rate = 0;
    double mem_limit_elems = 0;
    double job_groups = 1;  // batch groups per job: the cost weight of batch steps
    int anneal_iters = 0;   // order search: annealing moves applied to the winning tree
    // per-slice costing (size-targeted slicing: slices run a few at a time): sliced legs
    // add no version multiplicity, and a tensor above 2^cap_bits elements is penalised
    bool per_slice = false;
    int cap_bits = 0;
    bool parallel_greedy = false;  // greedy trials with their own generators, on threads
    int n_sliced = 0;              // |I|
    std::vector<int> idx_seg;      // segment id of each network index (-1: beta / other)
};

// Contraction tree node.
struct Node {
    Bits idx;              // network indices of the tensor
    uint64_t dep = 0;      // sliced edges its subtree depends on (bit e = I[e])
    int ch[2] = {-1, -1};  // children (internal nodes)
    int leaf = -1;         // leaf number (leaves)
    bool beta = false;     // carries beta bits (and no closed legs)
    std::vector<int> layout;  // storage order of idx, LSB first (set by the compiler)
};

// One pairwise contraction: C[v][bat][m][n] = sum_k A[v][bat][m][k] * B[v][bat][n][k].
struct Step {
    int c, a, b;                     // node ids, a = row operand
    int nbat, nm, nn, nk;            // bit counts
    int8_t pos_bat[64], pos_m[64], pos_n[64];  // bit positions in C's layout
    double flops_per_version;        // 8 * 2^(nbat+nm+nn+nk)
    // Batch gathers: operand o (0 = a, 1 = b) is stored with its closed legs as the top
    // g_nq[o] layout bits (closed positions g_q[o][0..], lowest first) and is read as
    // the operand layout in which the beta bits sit at positions g_pos_beta[o][0..]
    // (beta bit t) and the remaining stored bits fill the other positions in order.
    int8_t gat[2];
    int8_t g_nq[2];
    int16_t g_q[2][32];
    int8_t g_pos_beta[2][16];
    int8_t g_nbits[2];               // layout bits of the gathered operand
};

struct Tree {
    std::vector<Node> nodes;  // leaves first (node i = leaf i), then internal in SSA order
    int root = -1;
    int q_max = -2;           // batch-selection threshold the tree was built with (-2: the network's)
};

struct TreeCost {
    double flops = 0;     // algorithmic FLOPs over all versions
    double bytes = 0;     // operand + result bytes
    double time = 0;      // estimated seconds
    int log2_max = 0;     // largest per-version tensor (log2 elements)
    double max_versioned = 0;  // largest versioned tensor (elements)
};

// Planner entry points (planner.cpp).
struct MergedGate {
    int qa, qb, sa, sb;
    cplx M[16];  // index (oa<<3)|(ob<<2)|(ia<<1)|ib
};

struct Merged {
    int n = 0;
    std::vector<MergedGate> gates;
    std::vector<int> n2q;             // two-qubit gates per qubit
    std::vector<cplx> input;          // 2 per qubit: leading single-qubit gates applied to |0>
    std::vector<int> seg_base;        // segment id of (q, s) = seg_base[q] + s
    int n_seg = 0;
};

void tn_merge(const tn_circuit_s &c, Merged &mg);

// Alg. 2 on the merged view: returns S as positions into I (sorted by (qubit, segment)).
std::vector<int> tn_sliced_vertex_select(const Merged &mg, const std::vector<tn_edge> &I, int k);
// Lightcone union (merged gate ids) of a set of vertices.
std::vector<int> tn_lightcone(const Merged &mg, const std::vector<tn_edge> &S);

// Network of the amplitude batches: open legs, beta selector leaves, sliced legs.
int tn_build_amp_network(const Merged &mg, const std::vector<tn_edge> &I, const std::vector<int> &open,
                         int log2_batches, Network &net, std::vector<int> &closed_qubits);
// Norm network C1 (x) C1* (Fig. 1) with the S legs identified; output = S legs in S order.
int tn_build_norm_network(const Merged &mg, const std::vector<tn_edge> &S, Network &net);

// Contraction order and tree compilation.
void tn_tree_from_leaves(const Network &net, Tree &t);
void tn_tree_from_leaves(const Network &net, Tree &t, int q_max);
Bits tn_leaf_closed(const Network &net, int leaf);  // closed-output ids on a leaf's legs
int tn_tree_from_ssa(const Network &net, const int32_t *pairs, int n_pairs, Tree &t);
void tn_greedy_tree(const Network &net, uint64_t seed, int trials, Tree &best, TreeCost &cost);
// Recursive min-cut bisection order (one trial) and the combined search: greedy trials,
// plus bisection trials on networks of 48 leaves or more, over several batch-selection
// thresholds (Network::q_max) when the network has closed legs; lowest estimated time
// wins and net.q_max is set to the winner's threshold.
void tn_bisect_tree(const Network &net, uint64_t seed, double eps, int cutoff, Tree &t);
void tn_search_tree(Network &net, uint64_t seed, int trials, Tree &best, TreeCost &cost);
// Replace each subtree cut at up to k frontier tensors by its cheapest order (subset DP).
void tn_reconfigure_tree(const Network &net, Tree &t, int k, int passes);
void tn_anneal_tree(const Network &net, Tree &t, int iters, uint64_t seed);
TreeCost tn_tree_cost(const Network &net, const Tree &t);
void tn_recompute_deps(const Network &net, Tree &t);
std::vector<int> tn_auto_slice(const Merged &mg, Network &net, Tree &t, int n_slice);
// Slice until every tensor of one slice holds at most `target` indices (<= max_legs legs).
std::vector<int> tn_width_slice(Network &net, Tree &t, int target, int max_legs);
// Shapes run on the tensor cores in the split precisions: K >= 16 and either M, N >= 64,
// or one side >= 128 (the rows) and the other >= 32 (32-column tiles).
inline bool tn_tc_shape(int nm, int nn, int nk) {
    return nk >= 4 && ((nm >= 6 && nn >= 6) || (std::max(nm, nn) >= 7 && std::min(nm, nn) >= 5));
}
// Tensor-core shapes whose short side needs the rows on the long side.
inline bool tn_tc_narrow(int nm, int nn, int nk) { return tn_tc_shape(nm, nn, nk) && std::min(nm, nn) < 6; }

// Compile with explicit-version legs E (bit e = I[e]); every other sliced leg below a
// node is one more layout bit of that node (never summed until the root).  tc_roles:
// tensor-core shaped steps put C's lowest layout bit on the row (M) side, since their
// epilogue stores one row per thread; other steps put it on the column (N) side.
int tn_compile(const Network &net, Tree &t, uint64_t E, std::vector<Step> &steps, bool tc_roles = false);
Bits tn_node_bits(const Network &net, const Node &x, uint64_t E);

// Whole host-side planning: sliced edges (given or auto), the amplitude network, the
// contraction tree (given SSA order or seeded greedy) and the compiled steps.
int tn_plan_build_host(const Merged &mg, const tn_plan_opts &o, const int32_t *order, int n_order,
                       const tn_edge *sliced, int n_sliced, const std::vector<int> &open,
                       std::vector<tn_edge> &I, Network &net, Tree &tree, std::vector<Step> &steps,
                       std::vector<int> &closed, uint64_t *E_used);
// Greedy tree of a network (or the SSA order when given) + compile.
void tn_cost_settings(Network &net, const tn_plan_opts &o);
int tn_tree_and_compile(Network &net, const tn_plan_opts &o, const int32_t *order, int n_order,
                        const Tree *candidate, Tree &tree, std::vector<Step> &steps, uint64_t *E_used,
                        bool tc_roles = false);
