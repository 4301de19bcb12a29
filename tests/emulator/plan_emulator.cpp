// Host execution of a compiled contraction plan, for CPU tests of the planner and the step
// compiler (test infrastructure; nothing in the library uses it).  It builds the plan with
// the library's own host planner, compiles it for the explicit legs of a slice set, and
// runs every step of the step list as plain complex128 loops:
//   * leaves in the layout the compiler fixed, one copy per code of their explicit legs;
//   * operand versions selected by the slice set, as the engine's layout_call lists them;
//   * batch gathers by the bit-by-bit definition of the step's gather fields;
//   * C[v][bat][m][n] = sum_k A[v][bat][m][k] B[v][bat][n][k], stored at the bit-scattered
//     positions the step gives;
//   * batch-independent steps run in the first batch group only (the stem is reused);
//   * out[t][i] = sum over root versions and free version bits of the root, in FP64.
// Each tensor has its own storage, so the engine's arena placement is not emulated.
#include <cstdio>
#include <cstring>
#include <unordered_map>

#include "tn_internal.h"
#include "planner.cpp"
#include "arena.h"

static thread_local std::string g_err;
void tn_set_error(const std::string &m) { g_err = m; }
void tn_plan_opts_default(tn_plan_opts *o) {
    std::memset(o, 0, sizeof(*o));
    o->log2_batches = 8;
    o->order_trials = 64;
    o->job_groups = 1;
}

extern "C" const char *emu_error() { return g_err.c_str(); }


// Plan (options o, q_max forced when >= -1, tensor-core operand roles when tc != 0),
// compile for the slice set and contract nb batches: out[2 * (t * 2^n_open + i) + {0, 1}].
// sliced_out receives the plan's sliced edges (qubit, segment pairs; cap 64).
extern "C" int emu_contract(const void *circ, size_t len, const int32_t *open, int n_open, const tn_plan_opts *o,
                            int q_max, int tc, const uint64_t *slices, int n_slices, const uint64_t *closed_bits,
                            int64_t nb, double *out, int32_t *sliced_out, int32_t *n_sliced_out, int32_t *stats) {
    tn_circuit_s c;
    int rc = tn_parse_circuit(circ, len, &c);
    if (rc) return rc;
    Merged mg;
    tn_merge(c, mg);
    std::vector<int> openv(open, open + n_open), closed;
    std::vector<tn_edge> I;
    Network net;
    Tree tree;
    std::vector<Step> steps;
    uint64_t E0 = 0;
    rc = tn_plan_build_host(mg, *o, nullptr, 0, nullptr, 0, openv, I, net, tree, steps, closed, &E0);
    if (rc) return rc;
    if (q_max >= -1) {
        net.q_max = q_max;
        tree.q_max = q_max;
        tn_recompute_deps(net, tree);
    }
    *n_sliced_out = (int32_t)I.size();
    for (size_t e = 0; e < I.size() && e < 64; e++) {
        sliced_out[2 * e] = I[e].qubit;
        sliced_out[2 * e + 1] = I[e].segment;
    }
    const std::vector<uint64_t> sv(slices, slices + n_slices);
    const int nI = (int)I.size();
    const uint64_t E = explicit_legs(sv, nI);
    rc = tn_compile(net, tree, E, steps, tc != 0);
    if (rc) return rc;
    const auto &nodes = tree.nodes;
    const int NN = (int)nodes.size();
    int n_gather = 0, n_batch_steps = 0;
    for (const Step &s : steps) {
        n_gather += s.gat[0] + s.gat[1];
        n_batch_steps += nodes[s.c].beta;
    }
    stats[0] = n_gather;
    stats[1] = n_batch_steps;
    stats[2] = (int32_t)steps.size();

    // versions: the distinct projections of the slice set on a node's explicit legs, as the
    // engine's layout_call orders them
    CallLayout lay;
    layout_call(tree, steps, E, 16, sv, lay);
    const auto &vals = lay.vals;
    const auto &vidx = lay.index;
    // leaves: one copy per code of their explicit sliced legs, in their layout
    std::vector<std::vector<cplx>> store(NN);
    std::vector<std::vector<int>> leaf_sl(NN);  // explicit sliced legs (e), in leg order
    for (int i = 0; i < (int)net.leaves.size(); i++) {
        const Leaf &lf = net.leaves[i];
        const Node &nd = nodes[i];
        std::vector<int> slp;
        for (size_t l = 0; l < lf.kind.size(); l++)
            if (lf.kind[l] == LEG_SLICED && ((E >> lf.ref[l]) & 1)) {
                slp.push_back((int)l);
                leaf_sl[i].push_back(lf.ref[l]);
            }
        const int nd_bits = (int)nd.layout.size();
        std::vector<int> leg(nd_bits, -1);
        for (int t = 0; t < nd_bits; t++) {
            const int id = nd.layout[t];
            const bool vbit = id >= net.n_idx && id < net.n_idx + net.n_sliced;
            for (size_t l = 0; l < lf.kind.size(); l++) {
                if (lf.kind[l] == LEG_NET && lf.ref[l] == id) leg[t] = (int)l;
                if (vbit && lf.kind[l] == LEG_SLICED && lf.ref[l] == id - net.n_idx) leg[t] = (int)l;
            }
            if (leg[t] < 0) { g_err = "leaf layout index not found"; return TN_EINVAL; }
        }
        const long long total = 1LL << (nd_bits + slp.size());
        store[i].assign((size_t)total, 0);
        for (long long g = 0; g < total; g++) {
            const long long code = g >> nd_bits, e = g & ((1LL << nd_bits) - 1);
            long long src = 0;
            for (int t = 0; t < nd_bits; t++) src |= ((e >> t) & 1LL) << leg[t];
            for (size_t u = 0; u < slp.size(); u++) src |= ((code >> u) & 1LL) << slp[u];
            store[i][(size_t)g] = lf.data[(size_t)src];
        }
    }
    auto version_of = [&](int x, uint64_t w) -> long long {
        if (nodes[x].ch[0] < 0) {
            long long code = 0;
            for (size_t u = 0; u < leaf_sl[x].size(); u++) code |= (long long)((w >> leaf_sl[x][u]) & 1ull) << u;
            return code;
        }
        return (long long)vidx[x].at(w);
    };
    auto scatter = [](long long x, const int8_t *pos, int n) {
        long long r = 0;
        for (int i = 0; i < n; i++) r |= ((x >> i) & 1LL) << pos[i];
        return r;
    };
    const int lT = closed.empty() ? 0 : o->log2_batches;
    const long long T = 1LL << lT;
    const int nout = (int)net.out_layout.size();
    const long long NA = 1LL << n_open;
    for (long long g0 = 0; g0 < nb; g0 += T) {
        std::vector<uint64_t> cb((size_t)T, 0);
        for (long long t = 0; t < T && g0 + t < nb; t++) cb[(size_t)t] = closed_bits[g0 + t];
        for (const Step &s : steps) {
            if (g0 > 0 && !nodes[s.c].beta) continue;  // the stem of the first group is kept
            // gathered operands, by the definition of the step's gather fields
            std::vector<cplx> gathered[2];
            for (int o2 = 0; o2 < 2; o2++) {
                if (!s.gat[o2]) continue;
                const int x = o2 ? s.b : s.a;
                const long long nv = nodes[x].ch[0] < 0 ? 1LL << leaf_sl[x].size() : (long long)vals[x].size();
                const int nbits = s.g_nbits[o2], lb = net.n_beta, nr = nbits - lb;
                const long long sp = 1LL << nodes[x].layout.size(), dp = 1LL << nbits;
                if (sp != (1LL << (nr + s.g_nq[o2]))) { g_err = "gathered operand size mismatch"; return TN_EINVAL; }
                gathered[o2].assign((size_t)(nv * dp), 0);
                for (long long v = 0; v < nv; v++)
                    for (long long e = 0; e < dp; e++) {
                        long long beta = 0, rest = 0;
                        int rp = 0;
                        for (int p = 0; p < nbits; p++) {
                            int tb = -1;
                            for (int t = 0; t < lb; t++)
                                if (s.g_pos_beta[o2][t] == p) tb = t;
                            if (tb >= 0) beta |= ((e >> p) & 1LL) << tb;
                            else rest |= ((e >> p) & 1LL) << rp++;
                        }
                        long long sel = 0;
                        for (int q = 0; q < s.g_nq[o2]; q++) sel |= (long long)((cb[(size_t)beta] >> s.g_q[o2][q]) & 1ull) << q;
                        gathered[o2][(size_t)(v * dp + e)] = store[x][(size_t)(v * sp + ((sel << nr) | rest))];
                    }
            }
            auto base = [&](int o2, uint64_t w) -> const cplx * {
                const int x = o2 ? s.b : s.a;
                if (s.gat[o2]) return gathered[o2].data() + version_of(x, w) * (1LL << s.g_nbits[o2]);
                return store[x].data() + version_of(x, w) * (1LL << nodes[x].layout.size());
            };
            const long long csize = 1LL << nodes[s.c].layout.size();
            store[s.c].assign((size_t)(csize * (long long)vals[s.c].size()), 0);
            for (size_t v = 0; v < vals[s.c].size(); v++) {
                const cplx *A = base(0, vals[s.c][v] & nodes[s.a].dep & E);
                const cplx *B = base(1, vals[s.c][v] & nodes[s.b].dep & E);
                cplx *C = store[s.c].data() + v * csize;
                for (long long bat = 0; bat < (1LL << s.nbat); bat++)
                    for (long long m = 0; m < (1LL << s.nm); m++)
                        for (long long n = 0; n < (1LL << s.nn); n++) {
                            cplx acc = 0;
                            for (long long k = 0; k < (1LL << s.nk); k++)
                                acc += A[(((bat << s.nm) | m) << s.nk) + k] * B[(((bat << s.nn) | n) << s.nk) + k];
                            C[scatter(bat, s.pos_bat, s.nbat) + scatter(m, s.pos_m, s.nm) + scatter(n, s.pos_n, s.nn)] = acc;
                        }
            }
        }
        const int root = tree.root;
        const long long rsize = 1LL << nodes[root].layout.size();
        const int nfree = (int)nodes[root].layout.size() - nout;
        for (long long t = 0; t < T && g0 + t < nb; t++)
            for (long long i = 0; i < NA; i++) {
                cplx acc = 0;
                const long long e = (t << n_open) | i;
                for (size_t v = 0; v < vals[root].size(); v++)
                    for (long long f = 0; f < (1LL << nfree); f++) acc += store[root][(size_t)(v * rsize + ((f << nout) | e))];
                double *o2 = out + 2 * ((g0 + t) * NA + i);
                o2[0] = acc.real();
                o2[1] = acc.imag();
            }
    }
    return TN_OK;
}

// The engine's arena layout for the compiled plan and slice set, checked: tensors live in
// the same step never overlap (an internal tensor lives from the step that writes it to
// the step that reads it, the root to the end, a gathered operand for its own step); the
// stem kept for later batch groups overlaps no other tensor at any time; every range ends
// within arena_bytes.  Returns the number of violations (negative: planning failed).
extern "C" int emu_layout_check(const void *circ, size_t len, const int32_t *open, int n_open, const tn_plan_opts *o,
                                int q_max, int tc, const uint64_t *slices, int n_slices, int64_t *arena_out) {
    tn_circuit_s c;
    if (tn_parse_circuit(circ, len, &c)) return -1;
    Merged mg;
    tn_merge(c, mg);
    std::vector<int> openv(open, open + n_open), closed;
    std::vector<tn_edge> I;
    Network net;
    Tree tree;
    std::vector<Step> steps;
    uint64_t E0 = 0;
    if (tn_plan_build_host(mg, *o, nullptr, 0, nullptr, 0, openv, I, net, tree, steps, closed, &E0)) return -1;
    if (q_max >= -1) {
        net.q_max = q_max;
        tree.q_max = q_max;
        tn_recompute_deps(net, tree);
    }
    const std::vector<uint64_t> sv(slices, slices + n_slices);
    const uint64_t E = explicit_legs(sv, (int)I.size());
    if (tn_compile(net, tree, E, steps, tc != 0)) return -1;
    CallLayout L;
    layout_call(tree, steps, E, 8, sv, L);
    *arena_out = (int64_t)L.arena_bytes;
    const auto &nodes = tree.nodes;
    const int NN = (int)nodes.size(), S = (int)steps.size();
    auto bytes_of = [&](int x) { return (size_t)L.nver[x] * (size_t(1) << nodes[x].layout.size()) * 8; };
    auto nver_of = [&](int x) -> long long {
        return nodes[x].ch[0] >= 0 ? L.nver[x] : 1LL << __builtin_popcountll(nodes[x].dep & E);
    };
    std::vector<int> born(NN, -1), dies(NN, -1);
    std::vector<char> kept(NN, 0);
    for (int i = 0; i < S; i++) {
        const Step &s = steps[i];
        born[s.c] = i;
        for (int ch : {s.a, s.b}) {
            dies[ch] = i;
            if (nodes[ch].ch[0] >= 0 && !nodes[ch].beta && nodes[s.c].beta) kept[ch] = 1;
        }
    }
    dies[tree.root] = S;
    struct R { size_t lo, hi; int tag; };
    int bad = 0;
    auto overlap = [](const R &a, const R &b) { return a.lo < b.hi && b.lo < a.hi; };
    std::vector<R> kept_r, other_r;
    for (int x = 0; x < NN; x++)
        if (nodes[x].ch[0] >= 0 && born[x] >= 0) {
            const R r{L.off[x], L.off[x] + bytes_of(x), x};
            if (r.hi > L.arena_bytes) bad++;
            (kept[x] ? kept_r : other_r).push_back(r);
        }
    for (int i = 0; i < S; i++)
        for (int o2 = 0; o2 < 2; o2++)
            if (steps[i].gat[o2]) {
                const int x = o2 ? steps[i].b : steps[i].a;
                const R r{L.goff[i][o2], L.goff[i][o2] + (size_t)nver_of(x) * (size_t(1) << steps[i].g_nbits[o2]) * 8,
                          -1 - i};
                if (r.hi > L.arena_bytes) bad++;
                other_r.push_back(r);
            }
    for (const R &k : kept_r) {
        for (const R &k2 : kept_r)
            if (k.tag < k2.tag && overlap(k, k2)) bad++;
        for (const R &r : other_r)
            if (overlap(k, r)) bad++;
    }
    // per step: the tensors and gathered operands live in it are disjoint
    for (int i = 0; i < S; i++) {
        std::vector<R> live;
        for (int x = 0; x < NN; x++)
            if (nodes[x].ch[0] >= 0 && born[x] >= 0 && !kept[x] && born[x] <= i && i <= dies[x])
                live.push_back({L.off[x], L.off[x] + bytes_of(x), x});
        for (int o2 = 0; o2 < 2; o2++)
            if (steps[i].gat[o2]) {
                const int x = o2 ? steps[i].b : steps[i].a;
                live.push_back({L.goff[i][o2], L.goff[i][o2] + (size_t)nver_of(x) * (size_t(1) << steps[i].g_nbits[o2]) * 8,
                                -1 - i - 1000000 * o2});
            }
        for (size_t u = 0; u < live.size(); u++)
            for (size_t v = u + 1; v < live.size(); v++)
                if (overlap(live[u], live[v])) bad++;
    }
    return bad;
}
