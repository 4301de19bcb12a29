// Host-side planner of libtn: circuit parsing, the merged tensor network, the seeded
// greedy contraction order, slicing, SlicedVertexSelect (App. B Alg. 2), the norm
// network of Fig. 1, and the compiler that turns a contraction tree into pairwise
// steps C[v][bat][m][n] = sum_k A[v][bat][m][k] B[v][bat][n][k] with layouts chosen
// top-down so that every operand is read as a plain row-major matrix.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <random>
#include <set>
#include <unordered_map>

#include "tn_internal.h"

// ------------------------------------------------------------------ circuit

int tn_parse_circuit(const void *buf_, size_t len, tn_circuit_s *c) {
    const unsigned char *buf = static_cast<const unsigned char *>(buf_);
    if (!buf || len < 12 || std::memcmp(buf, "RQC1", 4) != 0) {
        tn_set_error("circuit: bad magic or short buffer");
        return TN_EINVAL;
    }
    uint32_t n, ng;
    std::memcpy(&n, buf + 4, 4);
    std::memcpy(&ng, buf + 8, 4);
    if (n == 0 || n > 64) {
        tn_set_error("circuit: qubit count must be in [1, 64]");
        return TN_EINVAL;
    }
    c->n = (int)n;
    c->gates.clear();
    c->gates.reserve(ng);
    size_t off = 12;
    for (uint32_t i = 0; i < ng; i++) {
        uint32_t h[3];
        if (off + 12 > len) { tn_set_error("circuit: truncated gate header"); return TN_EINVAL; }
        std::memcpy(h, buf + off, 12);
        off += 12;
        if (h[0] != 1 && h[0] != 2) { tn_set_error("circuit: gate arity must be 1 or 2"); return TN_EINVAL; }
        size_t d = size_t(1) << h[0];
        if (off + 16 * d * d > len) { tn_set_error("circuit: truncated gate matrix"); return TN_EINVAL; }
        TnGate g;
        g.arity = (int)h[0];
        g.q[0] = (int)h[1];
        g.q[1] = h[0] == 2 ? (int)h[2] : -1;
        if (h[1] >= n || (h[0] == 2 && (h[2] >= n || h[2] == h[1]))) {
            tn_set_error("circuit: qubit index out of range");
            return TN_EINVAL;
        }
        for (size_t e = 0; e < d * d; e++) {
            double re, im;
            std::memcpy(&re, buf + off + 16 * e, 8);
            std::memcpy(&im, buf + off + 16 * e + 8, 8);
            g.m[e] = cplx(re, im);
        }
        off += 16 * d * d;
        c->gates.push_back(g);
    }
    return TN_OK;
}

// ------------------------------------------------------------------ merged view

void tn_merge(const tn_circuit_s &c, Merged &mg) {
    const int n = c.n;
    mg.n = n;
    mg.gates.clear();
    mg.n2q.assign(n, 0);
    mg.input.assign(2 * n, cplx(0));
    for (int q = 0; q < n; q++) mg.input[2 * q] = 1.0;
    std::vector<std::array<cplx, 4>> pending(n, {cplx(1), cplx(0), cplx(0), cplx(1)});
    std::vector<int> last(n, -1);
    auto flush = [&](int w) {
        auto &P = pending[w];
        if (last[w] < 0) {
            cplx a0 = mg.input[2 * w], a1 = mg.input[2 * w + 1];
            mg.input[2 * w] = P[0] * a0 + P[1] * a1;
            mg.input[2 * w + 1] = P[2] * a0 + P[3] * a1;
        } else {
            MergedGate &g = mg.gates[last[w]];
            cplx out[16];
            const bool first = g.qa == w;
            for (int oa = 0; oa < 2; oa++)
                for (int ob = 0; ob < 2; ob++)
                    for (int ia = 0; ia < 2; ia++)
                        for (int ib = 0; ib < 2; ib++) {
                            cplx acc = 0;
                            for (int x = 0; x < 2; x++) {
                                if (first) acc += P[2 * oa + x] * g.M[(x << 3) | (ob << 2) | (ia << 1) | ib];
                                else acc += P[2 * ob + x] * g.M[(oa << 3) | (x << 2) | (ia << 1) | ib];
                            }
                            out[(oa << 3) | (ob << 2) | (ia << 1) | ib] = acc;
                        }
            std::memcpy(g.M, out, sizeof(out));
        }
        P = {cplx(1), cplx(0), cplx(0), cplx(1)};
    };
    for (const TnGate &g : c.gates) {
        if (g.arity == 1) {
            auto &P = pending[g.q[0]];
            std::array<cplx, 4> r;
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++) r[2 * i + j] = g.m[2 * i] * P[j] + g.m[2 * i + 1] * P[2 + j];
            P = r;
        } else {
            int a = g.q[0], b = g.q[1];
            flush(a);
            flush(b);
            MergedGate m;
            m.qa = a;
            m.qb = b;
            m.sa = mg.n2q[a];
            m.sb = mg.n2q[b];
            std::memcpy(m.M, g.m, sizeof(m.M));
            last[a] = last[b] = (int)mg.gates.size();
            mg.gates.push_back(m);
            mg.n2q[a]++;
            mg.n2q[b]++;
        }
    }
    for (int w = 0; w < n; w++) flush(w);
    mg.seg_base.assign(n, 0);
    int acc = 0;
    for (int q = 0; q < n; q++) {
        mg.seg_base[q] = acc;
        acc += mg.n2q[q] + 1;
    }
    mg.n_seg = acc;
}

// ------------------------------------------------------------------ lightcones

namespace {

struct Lightcones {
    const Merged &mg;
    std::map<std::pair<int, int>, int> producer;  // (q, s) -> merged gate whose output it is
    explicit Lightcones(const Merged &m) : mg(m) {
        for (int g = 0; g < (int)mg.gates.size(); g++) {
            const auto &x = mg.gates[g];
            producer[{x.qa, x.sa + 1}] = g;
            producer[{x.qb, x.sb + 1}] = g;
        }
    }
    void cone(std::pair<int, int> v, std::set<int> &out) const {
        std::vector<std::pair<int, int>> stack{v};
        while (!stack.empty()) {
            auto x = stack.back();
            stack.pop_back();
            auto it = producer.find(x);
            if (it == producer.end() || out.count(it->second)) continue;
            out.insert(it->second);
            const auto &g = mg.gates[it->second];
            stack.push_back({g.qa, g.sa});
            stack.push_back({g.qb, g.sb});
        }
    }
    std::set<std::pair<int, int>> inputs(const std::vector<std::pair<int, int>> &S) const {
        std::set<int> gates;
        for (auto &v : S) cone(v, gates);
        std::set<std::pair<int, int>> out;
        for (int g : gates) {
            out.insert({mg.gates[g].qa, mg.gates[g].sa});
            out.insert({mg.gates[g].qb, mg.gates[g].sb});
        }
        return out;
    }
};

}  // namespace

std::vector<int> tn_lightcone(const Merged &mg, const std::vector<tn_edge> &S) {
    Lightcones lc(mg);
    std::set<int> g;
    for (auto &v : S) lc.cone({v.qubit, v.segment}, g);
    return std::vector<int>(g.begin(), g.end());
}

// App. B Alg. 2 (SlicedVertexSelect).  Readings: the argmin runs over the candidate u;
// candidates exclude S itself; ties go to the earliest vertex of I; S is returned in
// (qubit, segment) order.
std::vector<int> tn_sliced_vertex_select(const Merged &mg, const std::vector<tn_edge> &I, int k) {
    Lightcones lc(mg);
    std::vector<std::pair<int, int>> S;
    std::vector<std::pair<int, int>> Iv;
    for (auto &e : I) Iv.push_back({e.qubit, e.segment});
    while ((int)S.size() < k) {
        auto lp = lc.inputs(S);
        int best = -1;
        size_t best_size = 0;
        for (int u = 0; u < (int)Iv.size(); u++) {
            if (lp.count(Iv[u])) continue;
            if (std::find(S.begin(), S.end(), Iv[u]) != S.end()) continue;
            auto S2 = S;
            S2.push_back(Iv[u]);
            size_t sz = lc.inputs(S2).size();
            if (best < 0 || sz < best_size) { best = u; best_size = sz; }
        }
        if (best < 0) break;
        auto lv = lc.inputs({Iv[best]});
        std::vector<std::pair<int, int>> next;
        for (auto &s : S)
            if (!lv.count(s)) next.push_back(s);
        next.push_back(Iv[best]);
        S.swap(next);
    }
    std::sort(S.begin(), S.end());
    std::vector<int> pos;
    for (auto &s : S)
        for (int u = 0; u < (int)Iv.size(); u++)
            if (Iv[u] == s) { pos.push_back(u); break; }
    return pos;
}

// ------------------------------------------------------------------ leaves

namespace {

// Contract leg t of a leaf with a vector v (2 entries) and drop the leg.
void absorb_vector(Leaf &L, int t, const cplx *v) {
    const int r = (int)L.kind.size();
    std::vector<cplx> out(size_t(1) << (r - 1));
    for (size_t e = 0; e < out.size(); e++) {
        size_t lo = e & ((size_t(1) << t) - 1), hi = (e >> t) << (t + 1);
        out[e] = L.data[hi | lo] * v[0] + L.data[hi | lo | (size_t(1) << t)] * v[1];
    }
    L.data.swap(out);
    L.kind.erase(L.kind.begin() + t);
    L.ref.erase(L.ref.begin() + t);
}

}  // namespace

int tn_build_amp_network(const Merged &mg, const std::vector<tn_edge> &I, const std::vector<int> &open,
                         int log2_batches, Network &net, std::vector<int> &closed_qubits) {
    const int n = mg.n;
    std::vector<int> open_pos(n, -1);
    for (int r = 0; r < (int)open.size(); r++) {
        if (open[r] < 0 || open[r] >= n || open_pos[open[r]] >= 0) {
            tn_set_error("plan: open qubits must be distinct and in range");
            return TN_EINVAL;
        }
        open_pos[open[r]] = r;
    }
    closed_qubits.clear();
    std::vector<int> closed_pos(n, -1);
    for (int q = 0; q < n; q++)
        if (open_pos[q] < 0) { closed_pos[q] = (int)closed_qubits.size(); closed_qubits.push_back(q); }
    std::vector<int> sliced_pos(mg.n_seg, -1);
    for (int e = 0; e < (int)I.size(); e++) {
        int q = I[e].qubit, s = I[e].segment;
        if (q < 0 || q >= n || s < 1 || s >= mg.n2q[q]) {
            tn_set_error("plan: sliced edge (" + std::to_string(q) + "," + std::to_string(s) +
                         ") is not an internal wire segment");
            return TN_EINVAL;
        }
        int id = mg.seg_base[q] + s;
        if (sliced_pos[id] >= 0) { tn_set_error("plan: duplicate sliced edge"); return TN_EINVAL; }
        sliced_pos[id] = e;
    }
    // network ids: every non-sliced internal segment and every open output
    std::vector<int> net_id(mg.n_seg, -1);
    int nid = 0;
    for (int q = 0; q < n; q++)
        for (int s = 1; s <= mg.n2q[q]; s++) {
            int id = mg.seg_base[q] + s;
            bool out = s == mg.n2q[q];
            if (out ? open_pos[q] >= 0 : sliced_pos[id] < 0) net_id[id] = nid++;
        }
    for (int q = 0; q < n; q++)
        if (mg.n2q[q] == 0 && open_pos[q] >= 0) net_id[mg.seg_base[q]] = nid++;
    net.n_beta = closed_qubits.empty() ? 0 : log2_batches;
    net.beta_base = nid;
    nid += net.n_beta;
    net.n_idx = nid;
    net.n_sliced = (int)I.size();
    if (nid > kMaxIdx) { tn_set_error("plan: network too large"); return TN_EUNSUPPORTED; }
    net.idx_seg.assign(nid, -1);
    for (int id = 0; id < mg.n_seg; id++)
        if (net_id[id] >= 0) net.idx_seg[net_id[id]] = id;
    net.leaves.clear();
    auto leg_of = [&](int q, int s, int &kind, int &ref) {
        int id = mg.seg_base[q] + s;
        bool out = s == mg.n2q[q];
        if (out && open_pos[q] < 0) { kind = LEG_CLOSED; ref = closed_pos[q]; }
        else if (!out && sliced_pos[id] >= 0) { kind = LEG_SLICED; ref = sliced_pos[id]; }
        else { kind = LEG_NET; ref = net_id[id]; }
    };
    for (const MergedGate &g : mg.gates) {
        Leaf L;
        L.data.assign(g.M, g.M + 16);
        // data bit 0 = in_b, 1 = in_a, 2 = out_b, 3 = out_a
        int segs[4][2] = {{g.qb, g.sb}, {g.qa, g.sa}, {g.qb, g.sb + 1}, {g.qa, g.sa + 1}};
        for (int t = 0; t < 4; t++) {
            int kind, ref;
            leg_of(segs[t][0], segs[t][1], kind, ref);
            L.kind.push_back(kind);
            L.ref.push_back(ref);
        }
        // absorb |0>-side vectors into input legs at segment 0 (higher leg first)
        if (g.sa == 0) absorb_vector(L, 1, &mg.input[2 * g.qa]);
        if (g.sb == 0) absorb_vector(L, 0, &mg.input[2 * g.qb]);
        net.leaves.push_back(std::move(L));
    }
    for (int q = 0; q < n; q++)
        if (mg.n2q[q] == 0) {
            Leaf L;
            L.data = {mg.input[2 * q], mg.input[2 * q + 1]};
            if (open_pos[q] >= 0) { L.kind = {LEG_NET}; L.ref = {net_id[mg.seg_base[q]]}; }
            else { L.kind = {LEG_CLOSED}; L.ref = {closed_pos[q]}; }
            net.leaves.push_back(std::move(L));
        }
    net.out_layout.clear();
    for (int r = 0; r < (int)open.size(); r++) net.out_layout.push_back(net_id[mg.seg_base[open[r]] + mg.n2q[open[r]]]);
    for (int t = 0; t < net.n_beta; t++) net.out_layout.push_back(net.beta_base + t);
    return TN_OK;
}

int tn_build_norm_network(const Merged &mg, const std::vector<tn_edge> &S, Network &net) {
    std::vector<int> gates = tn_lightcone(mg, S);
    std::set<int> in_c1(gates.begin(), gates.end());
    std::map<std::pair<int, int>, int> consumer;  // (q, s) consumed by a C1 gate
    for (int g : gates) {
        consumer[{mg.gates[g].qa, mg.gates[g].sa}] = g;
        consumer[{mg.gates[g].qb, mg.gates[g].sb}] = g;
    }
    std::map<std::pair<int, int>, int> s_pos;
    for (int t = 0; t < (int)S.size(); t++) s_pos[{S[t].qubit, S[t].segment}] = t;
    int nid = 0;
    // ids: shared S hyperedges first, then per-segment ket / bra / joint ids
    for (int t = 0; t < (int)S.size(); t++) nid++;
    std::map<std::pair<int, int>, int> ket_id, bra_id;
    auto id_of = [&](int q, int s, bool bra) -> int {
        auto key = std::make_pair(q, s);
        auto sp = s_pos.find(key);
        if (sp != s_pos.end()) return sp->second;
        bool internal = consumer.count(key) > 0;
        if (!internal) {  // a C1 output outside S: joined between C1 and C1*
            auto it = ket_id.find(key);
            if (it != ket_id.end()) return it->second;
            ket_id[key] = nid;
            return nid++;
        }
        auto &m = bra ? bra_id : ket_id;
        auto it = m.find(key);
        if (it != m.end()) return it->second;
        m[key] = nid;
        return nid++;
    };
    net.leaves.clear();
    for (int side = 0; side < 2; side++)
        for (int g : gates) {
            const MergedGate &x = mg.gates[g];
            Leaf L;
            for (int e = 0; e < 16; e++) L.data.push_back(side ? std::conj(x.M[e]) : x.M[e]);
            int segs[4][2] = {{x.qb, x.sb}, {x.qa, x.sa}, {x.qb, x.sb + 1}, {x.qa, x.sa + 1}};
            for (int t = 0; t < 4; t++) {
                L.kind.push_back(LEG_NET);
                L.ref.push_back(segs[t][1] == 0 ? -1 : id_of(segs[t][0], segs[t][1], side == 1));
            }
            std::vector<cplx> in_a(2), in_b(2);
            for (int r = 0; r < 2; r++) {
                in_a[r] = side ? std::conj(mg.input[2 * x.qa + r]) : mg.input[2 * x.qa + r];
                in_b[r] = side ? std::conj(mg.input[2 * x.qb + r]) : mg.input[2 * x.qb + r];
            }
            if (x.sa == 0) absorb_vector(L, 1, in_a.data());
            if (x.sb == 0) absorb_vector(L, 0, in_b.data());
            net.leaves.push_back(std::move(L));
        }
    net.n_idx = nid;
    net.n_beta = 0;
    net.beta_base = nid;
    net.n_sliced = 0;
    net.out_layout.clear();
    for (int t = 0; t < (int)S.size(); t++) net.out_layout.push_back(t);
    if (nid > kMaxIdx) { tn_set_error("norm network too large"); return TN_EUNSUPPORTED; }
    return TN_OK;
}

// ------------------------------------------------------------------ trees

void tn_tree_from_leaves(const Network &net, Tree &t) {
    t.nodes.clear();
    for (int i = 0; i < (int)net.leaves.size(); i++) {
        Node nd;
        nd.leaf = i;
        const Leaf &L = net.leaves[i];
        for (size_t l = 0; l < L.kind.size(); l++) {
            if (L.kind[l] == LEG_NET) nd.idx.set(L.ref[l]);
            else if (L.kind[l] == LEG_SLICED) nd.dep |= 1ull << L.ref[l];
            else nd.beta = true;
        }
        if (nd.beta)
            for (int b = 0; b < net.n_beta; b++) nd.idx.set(net.beta_base + b);
        t.nodes.push_back(nd);
    }
    t.root = t.nodes.size() == 1 ? 0 : -1;
}

namespace {

struct IdxCounts {
    std::vector<int> count;
    std::vector<char> out;
};

Node contract_nodes(const Node &a, const Node &b, const IdxCounts &ic) {
    Node c;
    Bits u = a.idx | b.idx, both = a.idx & b.idx;
    c.idx = u;
    for (int i : both.list())
        if (!ic.out[i] && ic.count[i] == 2) c.idx.clr(i);
    c.dep = a.dep | b.dep;
    c.beta = a.beta || b.beta;
    return c;
}

void counts_of(const Network &net, const std::vector<Node> &leaves, IdxCounts &ic) {
    ic.count.assign(net.n_idx, 0);
    ic.out.assign(net.n_idx, 0);
    for (int i : net.out_layout) ic.out[i] = 1;
    for (auto &nd : leaves)
        for (int i : nd.idx.list()) ic.count[i]++;
}

}  // namespace

int tn_tree_from_ssa(const Network &net, const int32_t *pairs, int n_pairs, Tree &t) {
    tn_tree_from_leaves(net, t);
    const int L = (int)t.nodes.size();
    if (n_pairs != L - 1) { tn_set_error("order: expected n_leaves-1 pairs"); return TN_EINVAL; }
    IdxCounts ic;
    counts_of(net, t.nodes, ic);
    std::vector<char> used(2 * L, 0);
    for (int p = 0; p < n_pairs; p++) {
        int a = pairs[2 * p], b = pairs[2 * p + 1];
        int cur = (int)t.nodes.size();
        if (a < 0 || b < 0 || a >= cur || b >= cur || a == b || used[a] || used[b]) {
            tn_set_error("order: invalid or reused tensor id in pair " + std::to_string(p));
            return TN_EINVAL;
        }
        used[a] = used[b] = 1;
        Node c = contract_nodes(t.nodes[a], t.nodes[b], ic);
        for (int i : (t.nodes[a].idx & t.nodes[b].idx).list()) ic.count[i] -= (c.idx.has(i) ? 1 : 2);
        c.ch[0] = a;
        c.ch[1] = b;
        t.nodes.push_back(c);
    }
    t.root = (int)t.nodes.size() - 1;
    return TN_OK;
}

void tn_recompute_deps(const Network &net, Tree &t) {
    Tree fresh;
    tn_tree_from_leaves(net, fresh);
    IdxCounts ic;
    counts_of(net, fresh.nodes, ic);
    for (size_t i = 0; i < fresh.nodes.size(); i++) {
        t.nodes[i].idx = fresh.nodes[i].idx;
        t.nodes[i].dep = fresh.nodes[i].dep;
        t.nodes[i].beta = fresh.nodes[i].beta;
    }
    for (size_t i = fresh.nodes.size(); i < t.nodes.size(); i++) {
        Node &c = t.nodes[i];
        const Node &a = t.nodes[c.ch[0]], &b = t.nodes[c.ch[1]];
        Node x = contract_nodes(a, b, ic);
        for (int j : (a.idx & b.idx).list()) ic.count[j] -= (x.idx.has(j) ? 1 : 2);
        c.idx = x.idx;
        c.dep = x.dep;
        c.beta = x.beta;
    }
}

TreeCost tn_tree_cost(const Network &net, const Tree &t) {
    (void)net;
    TreeCost tc;
    const double flop_rate = 50e12, bw = 5.5e12, launch = 4e-6;
    for (auto &nd : t.nodes) {
        int l = nd.idx.count();
        tc.log2_max = std::max(tc.log2_max, l);
        tc.max_versioned = std::max(tc.max_versioned, std::ldexp(1.0, l + __builtin_popcountll(nd.dep)));
        if (nd.ch[0] < 0) continue;
        const Node &a = t.nodes[nd.ch[0]], &b = t.nodes[nd.ch[1]];
        double ver = std::ldexp(1.0, __builtin_popcountll(nd.dep));
        double fl = 8.0 * std::ldexp(1.0, (a.idx | b.idx).count()) * ver;
        double by = 8.0 * (std::ldexp(1.0, a.idx.count() + __builtin_popcountll(a.dep)) +
                           std::ldexp(1.0, b.idx.count() + __builtin_popcountll(b.dep)) +
                           std::ldexp(1.0, l) * ver);
        tc.flops += fl;
        tc.bytes += by;
        tc.time += std::max(fl / flop_rate, by / bw) + launch;
    }
    return tc;
}

namespace {

// One randomised greedy pass (memory-removed score with Gumbel noise).
void greedy_once(const Network &net, std::mt19937_64 &rng, double costmod, double temperature, Tree &t) {
    tn_tree_from_leaves(net, t);
    const int L = (int)t.nodes.size();
    if (L == 1) { t.root = 0; return; }
    IdxCounts ic;
    counts_of(net, t.nodes, ic);
    std::vector<char> alive(2 * L, 0);
    for (int i = 0; i < L; i++) alive[i] = 1;
    std::set<std::pair<int, int>> pairs;
    {
        std::vector<std::vector<int>> by_idx(net.n_idx);
        for (int i = 0; i < L; i++)
            for (int j : t.nodes[i].idx.list()) by_idx[j].push_back(i);
        for (auto &v : by_idx)
            for (size_t x = 0; x < v.size(); x++)
                for (size_t y = x + 1; y < v.size(); y++) pairs.insert({v[x], v[y]});
    }
    std::uniform_real_distribution<double> U(1e-12, 1.0);
    auto lsize = [](const Node &x) { return x.idx.count() + __builtin_popcountll(x.dep); };
    int n_alive = L;
    while (n_alive > 1) {
        int ba = -1, bb = -1;
        double best = 0;
        if (pairs.empty()) {
            // disconnected: outer product of the two smallest
            std::vector<std::pair<int, int>> al;
            for (int i = 0; i < (int)t.nodes.size(); i++)
                if (alive[i]) al.push_back({lsize(t.nodes[i]), i});
            std::sort(al.begin(), al.end());
            ba = al[0].second;
            bb = al[1].second;
        } else {
            for (auto &pr : pairs) {
                const Node &a = t.nodes[pr.first], &b = t.nodes[pr.second];
                Node c = contract_nodes(a, b, ic);
                double sc = std::ldexp(1.0, lsize(c)), sa = std::ldexp(1.0, lsize(a)), sb = std::ldexp(1.0, lsize(b));
                double x = sc - costmod * (sa + sb);
                double key = (x >= 0 ? 1.0 : -1.0) * std::log2(1.0 + std::fabs(x));
                if (temperature > 0) key -= temperature * (-std::log(-std::log(U(rng))));
                if (ba < 0 || key < best) { best = key; ba = pr.first; bb = pr.second; }
            }
        }
        Node c = contract_nodes(t.nodes[ba], t.nodes[bb], ic);
        for (int j : (t.nodes[ba].idx & t.nodes[bb].idx).list()) ic.count[j] -= (c.idx.has(j) ? 1 : 2);
        c.ch[0] = ba;
        c.ch[1] = bb;
        int cid = (int)t.nodes.size();
        t.nodes.push_back(c);
        alive[ba] = alive[bb] = 0;
        alive[cid] = 1;
        n_alive--;
        for (auto it = pairs.begin(); it != pairs.end();) {
            if (it->first == ba || it->first == bb || it->second == ba || it->second == bb) it = pairs.erase(it);
            else ++it;
        }
        for (int d = 0; d < cid; d++)
            if (alive[d] && (t.nodes[d].idx & c.idx).any()) pairs.insert({d, cid});
    }
    t.root = (int)t.nodes.size() - 1;
}

}  // namespace

void tn_greedy_tree(const Network &net, uint64_t seed, int trials, Tree &best, TreeCost &cost) {
    std::mt19937_64 rng(seed * 0x9E3779B97F4A7C15ull + 12345);
    bool have = false;
    for (int tr = 0; tr < std::max(1, trials); tr++) {
        double costmod = tr == 0 ? 1.0 : std::uniform_real_distribution<double>(0.3, 2.0)(rng);
        double temp = tr == 0 ? 0.0 : std::uniform_real_distribution<double>(0.0, 1.5)(rng);
        Tree t;
        greedy_once(net, rng, costmod, temp, t);
        TreeCost c = tn_tree_cost(net, t);
        if (!have || c.time < cost.time) { best = t; cost = c; have = true; }
    }
}

// Slice network index `id` in a tree: it leaves every tensor, and every tensor above a
// leaf that held it gains dependence bit `bit`.
static void slice_tree(Tree &t, int id, int bit) {
    for (auto &nd : t.nodes) {
        if (nd.ch[0] < 0) {
            if (nd.idx.has(id)) { nd.idx.clr(id); nd.dep |= 1ull << bit; }
        } else {
            nd.idx.clr(id);
            nd.dep = t.nodes[nd.ch[0]].dep | t.nodes[nd.ch[1]].dep;
        }
    }
}

// Greedily slice n_slice more edges of the tree (each pick minimises the estimated time
// of the versioned contraction); moves them from network indices to sliced legs and
// returns the picked network ids.
std::vector<int> tn_auto_slice(const Merged &mg, Network &net, Tree &t, int n_slice) {
    (void)mg;
    std::vector<int> picked;
    std::vector<char> is_out(net.n_idx, 0);
    for (int i : net.out_layout) is_out[i] = 1;
    for (int r = 0; r < n_slice; r++) {
        std::vector<int> cnt(net.n_idx, 0);
        for (auto &L : net.leaves)
            for (size_t l = 0; l < L.kind.size(); l++)
                if (L.kind[l] == LEG_NET) cnt[L.ref[l]]++;
        int best = -1;
        TreeCost bestc;
        for (int id = 0; id < net.n_idx; id++) {
            if (cnt[id] != 2 || is_out[id]) continue;
            Tree tt = t;
            slice_tree(tt, id, net.n_sliced);
            TreeCost c = tn_tree_cost(net, tt);
            if (best < 0 || c.time < bestc.time ||
                (c.time == bestc.time && c.max_versioned < bestc.max_versioned)) { best = id; bestc = c; }
        }
        if (best < 0) break;
        for (auto &L : net.leaves)
            for (size_t l = 0; l < L.kind.size(); l++)
                if (L.kind[l] == LEG_NET && L.ref[l] == best) { L.kind[l] = LEG_SLICED; L.ref[l] = net.n_sliced; }
        slice_tree(t, best, net.n_sliced);
        net.n_sliced++;
        picked.push_back(best);
    }
    return picked;
}

// ------------------------------------------------------------------ compiler

// Layout bits of a node: its network indices plus one bit per sliced leg below it that
// is not an explicit version (a sliced leg whose values all appear in the slice set
// is carried like an index that is never summed until the root).
Bits tn_node_bits(const Network &net, const Node &x, uint64_t E) {
    Bits b = x.idx;
    uint64_t fr = x.dep & ~E;
    while (fr) {
        int e = __builtin_ctzll(fr);
        b.set(net.n_idx + e);
        fr &= fr - 1;
    }
    return b;
}

int tn_compile(const Network &net, Tree &t, uint64_t E, std::vector<Step> &steps, bool tc_roles) {
    steps.clear();
    if (net.n_idx + net.n_sliced > kMaxIdx) { tn_set_error("compile: index space too large"); return TN_EUNSUPPORTED; }
    Node &root = t.nodes[t.root];
    // the root's index set must equal the output set
    Bits outb;
    for (int i : net.out_layout) outb.set(i);
    if ((root.idx.andnot(outb)).any() || (outb.andnot(root.idx)).any()) {
        tn_set_error("compile: root indices differ from the output indices");
        return TN_EINVAL;
    }
    root.layout = net.out_layout;
    for (int e = 0; e < net.n_sliced; e++)
        if (((root.dep & ~E) >> e) & 1) root.layout.push_back(net.n_idx + e);
    for (auto &nd : t.nodes)
        if (tn_node_bits(net, nd, E).count() > 40) {
            tn_set_error("compile: tensor with more than 40 index bits");
            return TN_EUNSUPPORTED;
        }
    for (int ci = (int)t.nodes.size() - 1; ci >= 0; ci--) {
        Node &c = t.nodes[ci];
        if (c.ch[0] < 0) continue;
        int a = c.ch[0], b = c.ch[1];
        Bits Cb = tn_node_bits(net, c, E);
        if (c.layout.empty() && Cb.any()) { tn_set_error("compile: node without layout"); return TN_EINVAL; }
        Bits A = tn_node_bits(net, t.nodes[a], E), B = tn_node_bits(net, t.nodes[b], E);
        Bits bat = A & B & Cb, m = (A & Cb).andnot(B), nn = (B & Cb).andnot(A), k = (A & B).andnot(Cb);
        if (((A | B).andnot(Cb | k)).any() || (Cb.andnot(A | B)).any()) {
            tn_set_error("compile: dangling index");
            return TN_EINVAL;
        }
        // the operand holding most of C's lowest layout positions takes the side the
        // epilogue walks across threads (consecutive threads -> consecutive addresses):
        // columns for the FFMA kernels, rows for the tensor-core kernel
        const bool rows_side = tc_roles && tn_tc_shape(m.count(), nn.count(), k.count());
        {
            int cm = 0, cn = 0, first = 0;
            for (size_t q = 0; q < c.layout.size() && q < 5; q++) {
                if (m.has(c.layout[q])) { cm++; if (!first) first = 1; }
                if (nn.has(c.layout[q])) { cn++; if (!first) first = 2; }
            }
            const bool m_low = cm > cn || (cm == cn && first == 1);
            if (m_low != rows_side) { std::swap(a, b); std::swap(m, nn); }
        }
        auto in_c_order = [&](const Bits &s) {
            std::vector<int> v;
            for (int id : c.layout)
                if (s.has(id)) v.push_back(id);
            return v;
        };
        std::vector<int> vb = in_c_order(bat), vm = in_c_order(m), vn = in_c_order(nn), vk = k.list();
        // k bits are the lowest layout bits of both operands: group them by the child of
        // the larger internal operand they come from (larger group first), so that
        // operand's producer writes long contiguous runs along one of its sides
        {
            int x = -1;
            double best = -1;
            for (int o : {a, b})
                if (t.nodes[o].ch[0] >= 0) {
                    double sz = std::ldexp(1.0, tn_node_bits(net, t.nodes[o], E).count());
                    if (sz > best) { best = sz; x = o; }
                }
            if (x >= 0) {
                Bits X1 = tn_node_bits(net, t.nodes[t.nodes[x].ch[0]], E), X2 = tn_node_bits(net, t.nodes[t.nodes[x].ch[1]], E);
                std::vector<int> g1, g2, g3;
                for (int id : vk) {
                    if (X1.has(id) && !X2.has(id)) g1.push_back(id);
                    else if (X2.has(id) && !X1.has(id)) g2.push_back(id);
                    else g3.push_back(id);
                }
                if (g2.size() > g1.size()) std::swap(g1, g2);
                vk.clear();
                vk.insert(vk.end(), g1.begin(), g1.end());
                vk.insert(vk.end(), g2.begin(), g2.end());
                vk.insert(vk.end(), g3.begin(), g3.end());
            }
        }
        auto pos_in_c = [&](int id) {
            for (size_t p = 0; p < c.layout.size(); p++)
                if (c.layout[p] == id) return (int)p;
            return -1;
        };
        Step s;
        std::memset(&s, 0, sizeof(s));
        s.c = ci;
        s.a = a;
        s.b = b;
        s.nbat = (int)vb.size();
        s.nm = (int)vm.size();
        s.nn = (int)vn.size();
        s.nk = (int)vk.size();
        for (int i = 0; i < s.nbat; i++) s.pos_bat[i] = (int8_t)pos_in_c(vb[i]);
        for (int i = 0; i < s.nm; i++) s.pos_m[i] = (int8_t)pos_in_c(vm[i]);
        for (int i = 0; i < s.nn; i++) s.pos_n[i] = (int8_t)pos_in_c(vn[i]);
        s.flops_per_version = 8.0 * std::ldexp(1.0, s.nbat + s.nm + s.nn + s.nk);
        auto &la = t.nodes[a].layout;
        auto &lb = t.nodes[b].layout;
        la.clear();
        lb.clear();
        la.insert(la.end(), vk.begin(), vk.end());
        la.insert(la.end(), vm.begin(), vm.end());
        la.insert(la.end(), vb.begin(), vb.end());
        lb.insert(lb.end(), vk.begin(), vk.end());
        lb.insert(lb.end(), vn.begin(), vn.end());
        lb.insert(lb.end(), vb.begin(), vb.end());
        steps.push_back(s);
    }
    std::sort(steps.begin(), steps.end(), [](const Step &x, const Step &y) { return x.c < y.c; });
    return TN_OK;
}

// ------------------------------------------------------------------ whole plan

int tn_tree_and_compile(const Network &net, const tn_plan_opts &o, const int32_t *order, int n_order,
                        const Tree *candidate, Tree &tree, std::vector<Step> &steps, uint64_t *E_used,
                        bool tc_roles) {
    if (order) {
        int rc = tn_tree_from_ssa(net, order, n_order, tree);
        if (rc) return rc;
    } else {
        TreeCost tc;
        tn_greedy_tree(net, o.order_seed, o.order_trials > 0 ? o.order_trials : 64, tree, tc);
        if (candidate) {
            Tree cand = *candidate;
            tn_recompute_deps(net, cand);
            TreeCost cc = tn_tree_cost(net, cand);
            if (cc.time < tc.time) tree = cand;
        }
    }
    // default variant: every sliced leg as a layout bit (full slice sets); if a tensor
    // would exceed the addressable bits, every sliced leg is an explicit version instead
    uint64_t E = 0;
    int rc = tn_compile(net, tree, E, steps, tc_roles);
    if (rc == TN_EUNSUPPORTED && net.n_sliced > 0) {
        E = net.n_sliced >= 64 ? ~0ull : ((1ull << net.n_sliced) - 1);
        rc = tn_compile(net, tree, E, steps, tc_roles);
    }
    if (E_used) *E_used = E;
    return rc;
}

int tn_plan_build_host(const Merged &mg, const tn_plan_opts &o, const int32_t *order, int n_order,
                       const tn_edge *sliced, int n_sliced, const std::vector<int> &open,
                       std::vector<tn_edge> &I, Network &net, Tree &tree, std::vector<Step> &steps,
                       std::vector<int> &closed, uint64_t *E_used) {
    I.clear();
    Tree t0;
    bool have_t0 = false;
    if (sliced) {
        I.assign(sliced, sliced + n_sliced);
    } else if (o.n_auto_sliced > 0) {
        // order the unsliced network, slice it greedily, then re-order with the slices
        Network net0;
        int rc = tn_build_amp_network(mg, {}, open, o.log2_batches, net0, closed);
        if (rc) return rc;
        TreeCost tc0;
        tn_greedy_tree(net0, o.order_seed, o.order_trials > 0 ? o.order_trials : 64, t0, tc0);
        std::vector<int> picked = tn_auto_slice(mg, net0, t0, o.n_auto_sliced);
        for (int id : picked) {
            int seg = net0.idx_seg[id], q = 0;
            while (q + 1 < mg.n && mg.seg_base[q + 1] <= seg) q++;
            I.push_back(tn_edge{q, seg - mg.seg_base[q]});
        }
        have_t0 = true;
    }
    int rc = tn_build_amp_network(mg, I, open, o.log2_batches, net, closed);
    if (rc) return rc;
    return tn_tree_and_compile(net, o, order, n_order, have_t0 ? &t0 : nullptr, tree, steps, E_used,
                               o.precision != TN_PREC_C64);
}
