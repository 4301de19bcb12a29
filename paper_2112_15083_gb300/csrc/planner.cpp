// Host-side planner of libtn: circuit parsing, the merged tensor network, the seeded
// greedy contraction order, slicing, SlicedVertexSelect (App. B Alg. 2), the norm
// network of Fig. 1, and the compiler that turns a contraction tree into pairwise
// steps C[v][bat][m][n] = sum_k A[v][bat][m][k] B[v][bat][n][k] with layouts chosen
// top-down so that every operand is read as a plain row-major matrix.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <random>
#include <thread>
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
    net.closed_base = nid;
    net.n_closed = (int)closed_qubits.size();
    nid += net.n_closed;
    net.n_beta = closed_qubits.empty() ? 0 : log2_batches;
    net.beta_base = nid;
    nid += net.n_beta;
    net.n_idx = nid;
    net.q_max = log2_batches;
    net.n_sliced = (int)I.size();
    if (nid > kMaxIdx) { tn_set_error("plan: network too large"); return TN_EUNSUPPORTED; }
    net.idx_seg.assign(nid, -1);
    for (int id = 0; id < mg.n_seg; id++)
        if (net_id[id] >= 0) net.idx_seg[net_id[id]] = id;
    net.leaves.clear();
    auto leg_of = [&](int q, int s, int &kind, int &ref) {
        int id = mg.seg_base[q] + s;
        bool out = s == mg.n2q[q];
        if (out && open_pos[q] < 0) { kind = LEG_NET; ref = net.closed_base + closed_pos[q]; }
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
            else { L.kind = {LEG_NET}; L.ref = {net.closed_base + closed_pos[q]}; }
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
    net.closed_base = nid;
    net.n_closed = 0;
    net.n_sliced = 0;
    net.out_layout.clear();
    for (int t = 0; t < (int)S.size(); t++) net.out_layout.push_back(t);
    if (nid > kMaxIdx) { tn_set_error("norm network too large"); return TN_EUNSUPPORTED; }
    return TN_OK;
}

// ------------------------------------------------------------------ trees

Bits tn_leaf_closed(const Network &net, int leaf) {
    Bits q;
    const Leaf &L = net.leaves[leaf];
    for (size_t l = 0; l < L.kind.size(); l++)
        if (L.kind[l] == LEG_NET && L.ref[l] >= net.closed_base && L.ref[l] < net.closed_base + net.n_closed) q.set(L.ref[l]);
    return q;
}

void tn_tree_from_leaves(const Network &net, Tree &t, int q_max) {
    t.nodes.clear();
    Bits beta;
    for (int b = 0; b < net.n_beta; b++) beta.set(net.beta_base + b);
    for (int i = 0; i < (int)net.leaves.size(); i++) {
        Node nd;
        nd.leaf = i;
        const Leaf &L = net.leaves[i];
        for (size_t l = 0; l < L.kind.size(); l++) {
            if (L.kind[l] == LEG_NET) nd.idx.set(L.ref[l]);
            else if (L.kind[l] == LEG_SLICED) nd.dep |= 1ull << L.ref[l];
        }
        // negative threshold: a leaf with closed legs is read in batch form from the start
        const Bits q = tn_leaf_closed(net, i);
        if (q_max < 0 && q.any() && net.n_beta >= 0) {
            nd.beta = true;
            nd.idx = nd.idx.andnot(q) | beta;
        }
        t.nodes.push_back(nd);
    }
    t.root = t.nodes.size() == 1 ? 0 : -1;
}

void tn_tree_from_leaves(const Network &net, Tree &t) { tn_tree_from_leaves(net, t, net.q_max); }

namespace {

struct IdxCounts {
    std::vector<int> count;
    std::vector<char> out;
    Bits closed, beta;  // closed-output ids, beta ids
    int q_max = 0;
};

// Result of contracting a and b.  Batch selection: the result carries the beta bits
// instead of closed legs when an operand does or when it would hold more than q_max
// closed legs (see Network).
Node contract_nodes(const Node &a, const Node &b, const IdxCounts &ic) {
    Node c;
    Bits u = a.idx | b.idx, both = a.idx & b.idx;
    c.idx = u;
    for (int i : both.list())
        if (!ic.out[i] && ic.count[i] == 2) c.idx.clr(i);
    c.dep = a.dep | b.dep;
    c.beta = a.beta || b.beta || (ic.q_max >= 0 && (c.idx & ic.closed).count() > ic.q_max);
    if (c.beta) c.idx = c.idx.andnot(ic.closed) | ic.beta;
    return c;
}

// The root carries the batch bits whenever the network has closed legs.
void seal_root(Node &r, const IdxCounts &ic) {
    if (!r.beta && (r.idx & ic.closed).any()) {
        r.beta = true;
        r.idx = r.idx.andnot(ic.closed) | ic.beta;
    }
}

void counts_of(const Network &net, const std::vector<Node> &leaves, IdxCounts &ic) {
    ic.count.assign(net.n_idx, 0);
    ic.out.assign(net.n_idx, 0);
    for (int i : net.out_layout) ic.out[i] = 1;
    for (auto &nd : leaves)
        for (int i : nd.idx.list()) ic.count[i]++;
    ic.closed = Bits();
    ic.beta = Bits();
    for (int c = 0; c < net.n_closed; c++) ic.closed.set(net.closed_base + c);
    for (int t = 0; t < net.n_beta; t++) ic.beta.set(net.beta_base + t);
    ic.q_max = net.q_max;
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
    seal_root(t.nodes[t.root], ic);
    t.q_max = net.q_max;
    return TN_OK;
}

void tn_recompute_deps(const Network &net, Tree &t) {
    Tree fresh;
    tn_tree_from_leaves(net, fresh, t.q_max >= -1 ? t.q_max : net.q_max);
    IdxCounts ic;
    counts_of(net, fresh.nodes, ic);
    if (t.q_max >= -1) ic.q_max = t.q_max;
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
    if (t.root >= 0) seal_root(t.nodes[t.root], ic);
}

namespace {

// Estimated time, FLOPs and bytes of contracting a and b into c (see tn_tree_cost).
struct StepEst {
    double time, flops, bytes;
};
StepEst step_estimate(const Network &net, const Node &a, const Node &b, const Node &c, const Bits &closed,
                      const Bits &beta) {
    // FFMA complex64 rate, HBM bandwidth and per-launch overhead (GB300 measurements of
    // the kernels in this library); tensor-core shaped steps at net.tc_flop_rate
    const double flop_rate = 3e13, bw = 5.5e12, launch = 4e-6;
    // an operand with closed legs read by a batch step is gathered first
    const bool ga = (a.ch[0] < 0 && a.beta) || (c.beta && !a.beta && (a.idx & closed).any());
    const bool gb = (b.ch[0] < 0 && b.beta) || (c.beta && !b.beta && (b.idx & closed).any());
    const Bits A = ga && !a.beta ? a.idx.andnot(closed) | beta : a.idx;
    const Bits B = gb && !b.beta ? b.idx.andnot(closed) | beta : b.idx;
    const double va = net.per_slice ? 1.0 : std::ldexp(1.0, __builtin_popcountll(a.dep));
    const double vb = net.per_slice ? 1.0 : std::ldexp(1.0, __builtin_popcountll(b.dep));
    const double ver = net.per_slice ? 1.0 : std::ldexp(1.0, __builtin_popcountll(c.dep));
    const double fl = 8.0 * std::ldexp(1.0, (A | B).count()) * ver;
    const double sa = 8.0 * std::ldexp(1.0, A.count()) * va, sb = 8.0 * std::ldexp(1.0, B.count()) * vb;
    const double by = sa + sb + 8.0 * std::ldexp(1.0, c.idx.count()) * ver;
    double gt = 0;
    if (ga) gt += 2 * sa / bw + launch;
    if (gb) gt += 2 * sb / bw + launch;
    // the launch's GEMM dims: version bits are layout bits, batch dims when both operands
    // carry them, rows or columns when one does
    const Bits &C = c.idx;
    const int vab = __builtin_popcountll(a.dep & b.dep);
    const int nb = (A & B & C).count() + vab;
    const int nm = (A & C).andnot(B).count() + __builtin_popcountll(a.dep) - vab;
    const int nn = (B & C).andnot(A).count() + __builtin_popcountll(b.dep) - vab;
    const int nk = (A & B).andnot(C).count();
    const int lo = std::min(nm, nn), hi = std::max(nm, nn);
    // FFMA kernels lose most of their rate when one side of the product is short
    // (measured: ~7 TFLOP/s at 16 x 32 outputs per batch, ~5 at 4 x 32, ~1 at 4 x 16)
    double rate = lo >= 6   ? flop_rate
                  : hi >= 7 ? flop_rate / 2
                  : lo >= 4 ? flop_rate / 4
                  : hi >= 5 ? flop_rate / 6
                            : flop_rate / 16;
    // at most 8 x 32 outputs over K >= 1024: the long-K kernel streams the operands, so the
    // bytes bound it
    if (lo <= 3 && hi <= 6 && nk >= 10) {
        rate = flop_rate;
    }
    if (net.tc_flop_rate > 0 && tn_tc_shape(hi, lo, nk)) {
        rate = net.tc_flop_rate * (lo >= 6 ? 1.0 : 0.5);
        // a batch of products of one or two output tiles each pays the tile's pipeline
        // fill and epilogue per few MMAs (measured 55-90 TFLOP/s for 2^17-2^18 batches of
        // 128-256 x 32 outputs)
        if (nb > 0 && nm + nn <= 14) rate = net.tc_flop_rate * 0.15;
    }
    // FFMA tiles over K <= 8 write each output after a few multiply-adds: they reach about a
    // third of the copy bandwidth (measured 1.2-1.7 TB/s on (0,3,25,7) and (0,7,25,3))
    const bool tc_step = net.tc_flop_rate > 0 && tn_tc_shape(hi, lo, nk);
    const double bw_step = !tc_step && nk <= 3 && lo >= 4 && C.count() >= 30 ? bw / 3 : bw;
    StepEst e;
    e.flops = fl;
    e.bytes = by + (ga ? 2 * sa : 0) + (gb ? 2 * sb : 0);
    e.time = std::max(fl / rate, by / bw_step) + launch + gt;
    if (net.mem_limit_elems > 0 && by / 8.0 > net.mem_limit_elems) e.time += 1e6 * (by / 8.0 / net.mem_limit_elems);
    // a batch step runs once per group of the job, a batch-independent one once per job
    if (c.beta) e.time *= net.job_groups;
    if (net.cap_bits > 0) {
        const int over = std::max({a.idx.count(), b.idx.count(), c.idx.count()}) - net.cap_bits;
        if (over > 0) e.time += 1e6 * over;
    }
    return e;
}

void closed_beta_masks(const Network &net, Bits &closed, Bits &beta) {
    for (int c = 0; c < net.n_closed; c++) closed.set(net.closed_base + c);
    for (int b = 0; b < net.n_beta; b++) beta.set(net.beta_base + b);
}

}  // namespace

TreeCost tn_tree_cost(const Network &net, const Tree &t) {
    TreeCost tc;
    Bits closed, beta;
    closed_beta_masks(net, closed, beta);
    for (auto &nd : t.nodes) {
        int l = nd.idx.count();
        tc.log2_max = std::max(tc.log2_max, l);
        tc.max_versioned = std::max(tc.max_versioned, std::ldexp(1.0, l + __builtin_popcountll(nd.dep)));
        if (nd.ch[0] < 0) continue;
        const StepEst e = step_estimate(net, t.nodes[nd.ch[0]], t.nodes[nd.ch[1]], nd, closed, beta);
        tc.flops += e.flops;
        tc.bytes += e.bytes;
        tc.time += e.time;
    }
    return tc;
}

// Subtree reconfiguration: every subtree cut at up to `k` frontier tensors is replaced by
// the order of least estimated time over those tensors (dynamic programming over subsets),
// for a few passes.  The tree keeps its leaves and batch-selection threshold.
void tn_reconfigure_tree(const Network &net, Tree &t, int k, int passes) {
    if (t.nodes.size() < 3 || t.root < 0) return;
    k = std::max(3, std::min(k, 10));
    Bits closed, beta;
    closed_beta_masks(net, closed, beta);
    const int qmax = t.q_max >= -1 ? t.q_max : net.q_max;
    Bits outb;
    for (int i : net.out_layout) outb.set(i);
    for (int pass = 0; pass < passes; pass++) {
        bool improved = false;
        // internal nodes, root first (breadth-first)
        std::vector<int> order{t.root};
        for (size_t q = 0; q < order.size(); q++)
            for (int c : t.nodes[order[q]].ch)
                if (c >= 0 && t.nodes[c].ch[0] >= 0) order.push_back(c);
        for (int x : order) {
            // frontier: expand the largest internal frontier node until k tensors
            std::vector<int> fr{t.nodes[x].ch[0], t.nodes[x].ch[1]};
            std::vector<int> internal{x};
            while ((int)fr.size() < k) {
                int bi = -1;
                for (int i = 0; i < (int)fr.size(); i++)
                    if (t.nodes[fr[i]].ch[0] >= 0 &&
                        (bi < 0 || t.nodes[fr[i]].idx.count() > t.nodes[fr[bi]].idx.count()))
                        bi = i;
                if (bi < 0) break;
                const int y = fr[bi];
                internal.push_back(y);
                fr[bi] = t.nodes[y].ch[0];
                fr.push_back(t.nodes[y].ch[1]);
            }
            const int m = (int)fr.size();
            if (m < 3) continue;
            // current cost of the subtree
            double cur = 0;
            for (int y : internal)
                cur += step_estimate(net, t.nodes[t.nodes[y].ch[0]], t.nodes[t.nodes[y].ch[1]], t.nodes[y], closed, beta).time;
            // subset nodes
            const Node &X = t.nodes[x];
            const Bits ext = X.idx | closed | beta | outb;
            const bool is_root = x == t.root;
            const int full = (1 << m) - 1;
            std::vector<Node> sub(full + 1);
            std::vector<Bits> uni(full + 1);
            for (int S = 1; S <= full; S++) {
                const int lo = __builtin_ctz(S);
                const int rest = S & (S - 1);
                if (!rest) {
                    sub[S] = t.nodes[fr[lo]];
                    uni[S] = sub[S].idx;
                    continue;
                }
                uni[S] = uni[1 << lo] | uni[rest];
            }
            for (int S = 1; S <= full; S++) {
                if (!(S & (S - 1))) continue;
                Node nd;
                Bits others = uni[full & ~S];
                Bits u = uni[S];
                nd.idx = u & (ext | others);
                nd.dep = 0;
                bool anyb = false;
                for (int i = 0; i < m; i++)
                    if (S >> i & 1) {
                        nd.dep |= t.nodes[fr[i]].dep;
                        anyb = anyb || t.nodes[fr[i]].beta;
                    }
                nd.beta = anyb || (qmax >= 0 && (nd.idx & closed).count() > qmax) ||
                          (S == full && is_root && (nd.idx & closed).any());
                if (nd.beta) nd.idx = nd.idx.andnot(closed) | beta;
                nd.ch[0] = 0;  // internal marker for step_estimate
                sub[S] = nd;
            }
            std::vector<double> best(full + 1, 0.0);
            std::vector<int> split(full + 1, 0);
            for (int S = 1; S <= full; S++) {
                if (!(S & (S - 1))) continue;
                double bv = -1;
                int bl = 0;
                // each unordered split once: L holds the lowest element of S
                const int low = S & -S;
                for (int L = (S - 1) & S; L > 0; L = (L - 1) & S) {
                    if (!(L & low)) continue;
                    const int R = S ^ L;
                    Node a = sub[L], b = sub[R];
                    if (!(L & (L - 1))) a = t.nodes[fr[__builtin_ctz(L)]];
                    if (!(R & (R - 1))) b = t.nodes[fr[__builtin_ctz(R)]];
                    const double v = best[L] + best[R] + step_estimate(net, a, b, sub[S], closed, beta).time;
                    if (bv < 0 || v < bv) { bv = v; bl = L; }
                }
                best[S] = bv;
                split[S] = bl;
            }
            if (!(best[full] < cur * (1 - 1e-9))) continue;
            // rebuild the subtree on the same internal node ids (x stays its root)
            std::vector<int> pool(internal.begin() + 1, internal.end());
            std::function<int(int, int)> build = [&](int S, int id) -> int {
                if (!(S & (S - 1))) return fr[__builtin_ctz(S)];
                const int L = split[S], R = S ^ L;
                const int node = id >= 0 ? id : pool.back();
                if (id < 0) pool.pop_back();
                const int a = build(L, -1), b = build(R, -1);
                Node &nd = t.nodes[node];
                nd.idx = sub[S].idx;
                nd.dep = sub[S].dep;
                nd.beta = sub[S].beta;
                nd.ch[0] = a;
                nd.ch[1] = b;
                nd.leaf = -1;
                return node;
            };
            build(full, x);
            improved = true;
        }
        if (!improved) break;
    }
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
    seal_root(t.nodes[t.root], ic);
    t.q_max = net.q_max;
}

}  // namespace

template <typename F>
static void parallel_for(int n, F f);

void tn_greedy_tree(const Network &net, uint64_t seed, int trials, Tree &best, TreeCost &cost) {
    if (net.parallel_greedy && trials > 1) {
        // each trial draws from its own generator (seed, trial), so the trials run in
        // parallel and the result does not depend on the thread count
        const int n = trials;
        std::vector<Tree> tt((size_t)n);
        std::vector<double> tc((size_t)n);
        parallel_for(n, [&](int tr) {
            std::mt19937_64 r(seed * 0x9E3779B97F4A7C15ull + 12345 + 0x632BE59BD9B4E019ull * (uint64_t)tr);
            const double costmod = tr == 0 ? 1.0 : std::uniform_real_distribution<double>(0.3, 2.0)(r);
            const double temp = tr == 0 ? 0.0 : std::uniform_real_distribution<double>(0.0, 1.5)(r);
            greedy_once(net, r, costmod, temp, tt[tr]);
            tc[tr] = tn_tree_cost(net, tt[tr]).time;
        });
        int bi = 0;
        for (int tr = 1; tr < n; tr++)
            if (tc[tr] < tc[bi]) bi = tr;
        best = tt[bi];
        cost = tn_tree_cost(net, best);
        return;
    }
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

namespace {

// Recursive min-cut bisection of the network's hypergraph: vertices are the leaves,
// hyperedges the network indices other than the beta bits and the open outputs (each a
// one-bit leg).  Every bisection is a Fiduccia-Mattheyses refinement of a grown region
// under a random imbalance; parts at or below `cutoff` leaves are contracted greedily.
struct Bisector {
    const Network &net;
    Tree &t;
    IdxCounts ic;
    std::mt19937_64 &rng;
    double eps;
    int cutoff;
    std::vector<std::vector<int>> vedges;  // leaf -> hyperedges
    std::vector<std::vector<int>> epins;   // hyperedge -> leaves

    Bisector(const Network &n, Tree &tree, std::mt19937_64 &r, double e, int c) : net(n), t(tree), rng(r), eps(e), cutoff(c) {
        tn_tree_from_leaves(net, t);
        counts_of(net, t.nodes, ic);
        const int L = (int)t.nodes.size();
        vedges.assign(L, {});
        epins.assign(net.n_idx, {});
        for (int v = 0; v < L; v++)
            for (int i : t.nodes[v].idx.list())
                if (!ic.out[i] && (net.n_beta == 0 || i < net.beta_base || i >= net.beta_base + net.n_beta)) {
                    vedges[v].push_back(i);
                    epins[i].push_back(v);
                }
    }

    int contract(int a, int b) {
        Node c = contract_nodes(t.nodes[a], t.nodes[b], ic);
        for (int j : (t.nodes[a].idx & t.nodes[b].idx).list()) ic.count[j] -= (c.idx.has(j) ? 1 : 2);
        c.ch[0] = a;
        c.ch[1] = b;
        t.nodes.push_back(c);
        return (int)t.nodes.size() - 1;
    }

    // Greedy pairwise contraction of the given nodes (smallest result growth first).
    int greedy(std::vector<int> alive) {
        auto lsize = [](const Node &x) { return x.idx.count() + __builtin_popcountll(x.dep); };
        while (alive.size() > 1) {
            int ba = -1, bb = -1;
            double best = 0;
            bool best_shared = false;
            for (size_t x = 0; x < alive.size(); x++)
                for (size_t y = x + 1; y < alive.size(); y++) {
                    const Node &a = t.nodes[alive[x]], &b = t.nodes[alive[y]];
                    bool shared = (a.idx & b.idx).andnot(ic.beta).any();
                    if (best_shared && !shared) continue;
                    Node c = contract_nodes(a, b, ic);
                    double key = std::ldexp(1.0, lsize(c)) - std::ldexp(1.0, lsize(a)) - std::ldexp(1.0, lsize(b));
                    if (ba < 0 || (shared && !best_shared) || key < best) {
                        best = key; ba = (int)x; bb = (int)y; best_shared = shared;
                    }
                }
            int c = contract(alive[ba], alive[bb]);
            alive.erase(alive.begin() + bb);
            alive[ba] = c;
        }
        return alive[0];
    }

    // FM bisection of `verts`: side[i] for verts[i]; returns the cut size.
    int bisect(const std::vector<int> &verts, std::vector<char> &side) {
        const int n = (int)verts.size();
        std::unordered_map<int, int> local;
        for (int i = 0; i < n; i++) local[verts[i]] = i;
        // hyperedges with at least two pins inside
        std::vector<std::vector<int>> ep;
        std::vector<std::vector<int>> ve(n);
        {
            std::unordered_map<int, int> eid;
            for (int i = 0; i < n; i++)
                for (int e : vedges[verts[i]]) {
                    int inside = 0;
                    for (int v : epins[e]) inside += local.count(v) ? 1 : 0;
                    if (inside < 2) continue;
                    auto it = eid.find(e);
                    int k;
                    if (it == eid.end()) { k = (int)ep.size(); eid[e] = k; ep.push_back({}); }
                    else k = it->second;
                    ep[k].push_back(i);
                    ve[i].push_back(k);
                }
        }
        const int lo = std::max(1, (int)std::floor(n * (1.0 - eps) / 2.0)), hi = std::min(n - 1, (int)std::ceil(n * (1.0 + eps) / 2.0));
        int best_cut = -1;
        std::vector<char> best_side;
        for (int start = 0; start < 3; start++) {
            // grow a connected region from a random vertex to n/2
            std::vector<char> s(n, 1);
            int size0 = 0;
            std::vector<int> queue{(int)(rng() % n)};
            std::vector<char> seen(n, 0);
            seen[queue[0]] = 1;
            size_t qh = 0;
            while (size0 < n / 2) {
                if (qh == queue.size()) {
                    int r = (int)(rng() % n);
                    while (seen[r]) r = (r + 1) % n;
                    seen[r] = 1;
                    queue.push_back(r);
                }
                int v = queue[qh++];
                s[v] = 0;
                size0++;
                std::vector<int> nb;
                for (int e : ve[v])
                    for (int u : ep[e])
                        if (!seen[u]) { seen[u] = 1; nb.push_back(u); }
                std::shuffle(nb.begin(), nb.end(), rng);
                queue.insert(queue.end(), nb.begin(), nb.end());
            }
            // FM passes
            std::vector<std::array<int, 2>> cnt(ep.size(), {0, 0});
            auto recount = [&]() {
                for (size_t e = 0; e < ep.size(); e++) {
                    cnt[e] = {0, 0};
                    for (int v : ep[e]) cnt[e][s[v]]++;
                }
            };
            auto cut_of = [&]() {
                int c = 0;
                for (size_t e = 0; e < ep.size(); e++) c += (cnt[e][0] > 0 && cnt[e][1] > 0);
                return c;
            };
            recount();
            int cut = cut_of();
            for (int pass = 0; pass < 8; pass++) {
                std::vector<int> gain(n, 0);
                for (int v = 0; v < n; v++)
                    for (int e : ve[v]) {
                        if (cnt[e][s[v]] == 1) gain[v]++;
                        if (cnt[e][1 - s[v]] == 0) gain[v]--;
                    }
                std::vector<char> locked(n, 0);
                std::vector<int> moves;
                int cur = cut, best_here = cut, best_len = 0, sz0 = 0;
                for (int v = 0; v < n; v++) sz0 += s[v] == 0;
                for (int step = 0; step < n; step++) {
                    int pick = -1;
                    for (int v = 0; v < n; v++) {
                        if (locked[v]) continue;
                        int nsz0 = sz0 + (s[v] == 0 ? -1 : 1);
                        if (nsz0 < lo || nsz0 > hi) continue;
                        if (pick < 0 || gain[v] > gain[pick] || (gain[v] == gain[pick] && (rng() & 1))) pick = v;
                    }
                    if (pick < 0) break;
                    int from = s[pick], to = 1 - from;
                    // update neighbour gains (classic FM bookkeeping, recomputed per edge)
                    for (int e : ve[pick]) {
                        for (int u : ep[e])
                            if (u != pick) {
                                if (cnt[e][s[u]] == 1) gain[u]--;
                                if (cnt[e][1 - s[u]] == 0) gain[u]++;
                            }
                        cnt[e][from]--;
                        cnt[e][to]++;
                        for (int u : ep[e])
                            if (u != pick) {
                                if (cnt[e][s[u]] == 1) gain[u]++;
                                if (cnt[e][1 - s[u]] == 0) gain[u]--;
                            }
                    }
                    cur -= gain[pick];
                    s[pick] = (char)to;
                    sz0 += to == 0 ? 1 : -1;
                    locked[pick] = 1;
                    moves.push_back(pick);
                    if (cur < best_here) { best_here = cur; best_len = (int)moves.size(); }
                }
                for (int m = (int)moves.size() - 1; m >= best_len; m--) s[moves[m]] = (char)(1 - s[moves[m]]);
                recount();
                int newcut = cut_of();
                if (newcut >= cut) { cut = newcut; break; }
                cut = newcut;
            }
            if (best_cut < 0 || cut < best_cut) { best_cut = cut; best_side = s; }
        }
        side = best_side;
        return best_cut;
    }

    int build(const std::vector<int> &verts) {
        if ((int)verts.size() <= cutoff) return greedy(verts);
        std::vector<char> side;
        bisect(verts, side);
        std::vector<int> p0, p1;
        for (size_t i = 0; i < verts.size(); i++) (side[i] ? p1 : p0).push_back(verts[i]);
        if (p0.empty() || p1.empty()) return greedy(verts);
        int a = build(p0), b = build(p1);
        return contract(a, b);
    }
};

}  // namespace

void tn_bisect_tree(const Network &net, uint64_t seed, double eps, int cutoff, Tree &t) {
    std::mt19937_64 rng(seed * 0xD1B54A32D192ED03ull + 777);
    Bisector b(net, t, rng, eps, cutoff);
    const int L = (int)t.nodes.size();
    if (L == 1) { t.root = 0; return; }
    std::vector<int> all(L);
    for (int i = 0; i < L; i++) all[i] = i;
    t.root = b.build(all);
    seal_root(t.nodes[t.root], b.ic);
    t.q_max = net.q_max;
}

namespace {

// The tree rebuilt in SSA order after its subtrees were reconfigured (net.q_max must be
// the tree's threshold).
bool reconfigured(const Network &net, const Tree &t, Tree &out) {
    Tree r = t;
    tn_reconfigure_tree(net, r, 6, 3);
    tn_reconfigure_tree(net, r, 8, 2);
    std::vector<int32_t> pairs;
    const int L = (int)net.leaves.size();
    std::vector<int> newid(r.nodes.size(), -1);
    for (int i = 0; i < L; i++) newid[i] = i;
    int next = L;
    std::function<void(int)> post = [&](int x) {
        if (r.nodes[x].ch[0] < 0) return;
        post(r.nodes[x].ch[0]);
        post(r.nodes[x].ch[1]);
        pairs.push_back(newid[r.nodes[x].ch[0]]);
        pairs.push_back(newid[r.nodes[x].ch[1]]);
        newid[x] = next++;
    };
    post(r.root);
    return tn_tree_from_ssa(net, pairs.data(), (int)pairs.size() / 2, out) == TN_OK;
}

}  // namespace

// f(i) for every i in [0, n), on up to hardware_concurrency() threads (thread w takes
// i = w, w + threads, ...).  Callers write results by index and combine them in index
// order, so the outcome does not depend on the thread count.
template <typename F>
static void parallel_for(int n, F f) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::min(std::min(hw, 32), n);
    if (nt <= 1) {
        for (int i = 0; i < n; i++) f(i);
        return;
    }
    std::vector<std::thread> th;
    th.reserve((size_t)nt);
    for (int w = 0; w < nt; w++)
        th.emplace_back([&f, w, nt, n] {
            for (int i = w; i < n; i += nt) f(i);
        });
    for (auto &x : th) x.join();
}

// Simulated annealing of the tree's shape: rotations x = (y, z), y = (a, b) -> x = (a, (b, z))
// or (b, (a, z)) at random internal nodes, accepted by the Metropolis rule on the log of the
// estimated time, with the temperature falling geometrically from 0.3 to 0.003 over `iters`
// moves.  Every candidate is rebuilt in SSA order (so its indices, batch flags and versions
// are exact for the threshold net.q_max); the cheapest tree seen replaces t.
void tn_anneal_tree(const Network &net, Tree &t, int iters, uint64_t seed) {
    const int L = (int)net.leaves.size();
    if (iters <= 0 || t.root < 0 || L < 4) return;
    std::vector<std::array<int, 2>> ch(t.nodes.size());
    for (size_t x = 0; x < t.nodes.size(); x++) ch[x] = {t.nodes[x].ch[0], t.nodes[x].ch[1]};
    const int root = t.root;
    auto rebuild = [&](Tree &out) -> bool {
        std::vector<int> order;  // internal nodes in post-order
        std::vector<std::pair<int, int>> stk{{root, 0}};
        while (!stk.empty()) {
            const int x = stk.back().first, st = stk.back().second;
            if (x < L) { stk.pop_back(); continue; }
            if (st < 2) {
                stk.back().second = st + 1;
                stk.push_back({ch[x][st], 0});
                continue;
            }
            order.push_back(x);
            stk.pop_back();
        }
        std::vector<int> newid(ch.size(), -1);
        for (int i = 0; i < L; i++) newid[i] = i;
        std::vector<int32_t> pairs;
        int next = L;
        for (int x : order) {
            pairs.push_back(newid[ch[x][0]]);
            pairs.push_back(newid[ch[x][1]]);
            newid[x] = next++;
        }
        return tn_tree_from_ssa(net, pairs.data(), (int)pairs.size() / 2, out) == TN_OK;
    };
    std::mt19937_64 rng(seed * 0x9E3779B97F4A7C15ull + 4242);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    double cur = tn_tree_cost(net, t).time, best_cost = cur;
    Tree best = t;
    const int n_int = (int)ch.size() - L;
    for (int it = 0; it < iters; it++) {
        const double temp = 0.3 * std::pow(0.01, (double)it / iters);
        int x = -1;
        for (int tries = 0; tries < 64 && x < 0; tries++) {
            const int c = L + (int)(rng() % (uint64_t)n_int);
            if (ch[c][0] >= L || ch[c][1] >= L) x = c;
        }
        if (x < 0) break;
        int side = ch[x][0] >= L ? 0 : 1;
        if (ch[x][0] >= L && ch[x][1] >= L) side = (int)(rng() & 1);
        const int y = ch[x][side], z = ch[x][1 - side];
        const int r = (int)(rng() & 1);
        const std::array<int, 2> old_x = ch[x], old_y = ch[y];
        ch[y] = {old_y[1 - r], z};
        ch[x] = {old_y[r], y};
        Tree cand;
        const bool ok = rebuild(cand);
        const double c = ok ? tn_tree_cost(net, cand).time : 0.0;
        const double d = ok ? std::log(c) - std::log(cur) : 1e300;
        if (ok && (d <= 0 || U(rng) < std::exp(-d / temp))) {
            cur = c;
            if (c < best_cost) { best_cost = c; best = cand; }
        } else {
            ch[x] = old_x;
            ch[y] = old_y;
        }
    }
    t = best;
}

void tn_search_tree(Network &net, uint64_t seed, int trials, Tree &best, TreeCost &cost) {
    // batch-selection thresholds to try: -1 (leaves with closed legs in batch form from
    // the start; all trials), then log2 T / 2 and log2 T (half the trials each)
    std::vector<int> qs{net.q_max};
    if (net.n_closed > 0 && net.n_beta > 0) qs = {-1, net.n_beta / 2, net.n_beta};
    std::mt19937_64 rng(seed * 0x9E3779B97F4A7C15ull + 99991);
    bool have = false;
    int best_q = net.q_max;
    for (size_t qi = 0; qi < qs.size(); qi++) {
        const int q = qs[qi], n = qi == 0 ? trials : std::max(1, trials / 2);
        net.q_max = q;
        // the few best greedy and bisection trees at this threshold ...
        std::vector<std::pair<double, Tree>> top;
        auto keep = [&](const Tree &t, double time) {
            if (top.size() < 3 || time < top.back().first) {
                top.emplace_back(time, t);
                std::sort(top.begin(), top.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
                if (top.size() > 3) top.pop_back();
            }
        };
        {
            Tree tg;
            TreeCost cg;
            tn_greedy_tree(net, seed + 131 * (q + 1), n, tg, cg);
            keep(tg, cg.time);
        }
        // (networks large enough for the greedy to go wrong also get bisection trials; their
        // parameters are drawn in trial order, the trials run in parallel)
        if (net.leaves.size() >= 48) {
            std::vector<double> eps((size_t)n);
            std::vector<int> cutoff((size_t)n);
            std::vector<uint64_t> tseed((size_t)n);
            for (int tr = 0; tr < n; tr++) {
                eps[tr] = std::uniform_real_distribution<double>(0.02, 0.6)(rng);
                cutoff[tr] = 4 + (int)(rng() % 24);
                tseed[tr] = rng();
            }
            std::vector<Tree> tb((size_t)n);
            std::vector<double> tt((size_t)n);
            const Network &cnet = net;
            parallel_for(n, [&](int tr) {
                tn_bisect_tree(cnet, tseed[tr], eps[tr], cutoff[tr], tb[tr]);
                tt[tr] = tn_tree_cost(cnet, tb[tr]).time;
            });
            for (int tr = 0; tr < n; tr++) keep(tb[tr], tt[tr]);
        }
        // ... each improved locally (optimal orders of its small subtrees), then compared
        std::vector<Tree> tq(top.size());
        std::vector<TreeCost> cq(top.size());
        const Network &cnet = net;
        parallel_for((int)top.size(), [&](int i) {
            tq[i] = top[i].second;
            cq[i] = tn_tree_cost(cnet, tq[i]);
            if (tq[i].nodes.size() >= 4) {
                Tree r;
                if (reconfigured(cnet, tq[i], r)) {
                    const TreeCost cr = tn_tree_cost(cnet, r);
                    if (cr.time < cq[i].time) { tq[i] = r; cq[i] = cr; }
                }
            }
        });
        for (size_t i = 0; i < top.size(); i++)
            if (!have || cq[i].time < cost.time) { best = tq[i]; cost = cq[i]; best_q = q; have = true; }
    }
    net.q_max = best_q;
    // optional: anneal the winner's shape from 8 independent seeds (in parallel), reconfigure
    // each result's small subtrees again, and keep the cheapest (first in seed order on ties)
    if (net.anneal_iters > 0 && have) {
        constexpr int kRestarts = 8;
        std::vector<Tree> a((size_t)kRestarts, best);
        std::vector<double> ta((size_t)kRestarts, 0.0);
        const Network &cnet = net;
        parallel_for(kRestarts, [&](int i) {
            tn_anneal_tree(cnet, a[i], cnet.anneal_iters, seed + 7919 * (uint64_t)i);
            Tree r;
            if (a[i].nodes.size() >= 4 && reconfigured(cnet, a[i], r) &&
                tn_tree_cost(cnet, r).time < tn_tree_cost(cnet, a[i]).time)
                a[i] = r;
            ta[i] = tn_tree_cost(cnet, a[i]).time;
        });
        for (int i = 0; i < kRestarts; i++)
            if (ta[i] < cost.time) { best = a[i]; cost = tn_tree_cost(net, a[i]); }
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

// Slice legs until no tensor of the tree holds more than `target` network indices (the
// per-version size, so that one slice's tensors fit in memory); each pick is the index
// held by the most oversized tensors, weighted by 2^(excess bits).  Returns the picked
// network ids (moved to sliced legs).
std::vector<int> tn_width_slice(Network &net, Tree &t, int target, int max_legs) {
    std::vector<int> picked;
    std::vector<char> is_out(net.n_idx, 0);
    for (int i : net.out_layout) is_out[i] = 1;
    while ((int)picked.size() < max_legs) {
        int maxb = 0;
        for (auto &nd : t.nodes) maxb = std::max(maxb, nd.idx.count());
        if (maxb <= target) break;
        std::vector<int> cnt(net.n_idx, 0);
        for (auto &L : net.leaves)
            for (size_t l = 0; l < L.kind.size(); l++)
                if (L.kind[l] == LEG_NET) cnt[L.ref[l]]++;
        std::vector<double> score(net.n_idx, 0.0);
        for (auto &nd : t.nodes) {
            const int b = nd.idx.count();
            if (b <= target) continue;
            const double w = std::ldexp(1.0, b - target);
            for (int id : nd.idx.list())
                if (cnt[id] == 2 && !is_out[id]) score[id] += w;
        }
        int best = -1;
        for (int id = 0; id < net.n_idx; id++)
            if (score[id] > 0 && (best < 0 || score[id] > score[best])) best = id;
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
    Bits closed, beta;
    for (int q = 0; q < net.n_closed; q++) closed.set(net.closed_base + q);
    for (int q = 0; q < net.n_beta; q++) beta.set(net.beta_base + q);
    if (t.nodes[t.root].ch[0] < 0 && net.n_closed > 0) {
        tn_set_error("compile: a single-tensor network with closed outputs");
        return TN_EUNSUPPORTED;
    }
    for (int ci = (int)t.nodes.size() - 1; ci >= 0; ci--) {
        Node &c = t.nodes[ci];
        if (c.ch[0] < 0) continue;
        int a = c.ch[0], b = c.ch[1];
        Bits Cb = tn_node_bits(net, c, E);
        if (c.layout.empty() && Cb.any()) { tn_set_error("compile: node without layout"); return TN_EINVAL; }
        Bits A = tn_node_bits(net, t.nodes[a], E), B = tn_node_bits(net, t.nodes[b], E);
        // operands with closed legs read by a batch step are gathered: they enter the
        // step with the beta bits in place of their closed legs
        // (a leaf in batch form from the start is stored with its closed legs and gathered)
        const bool leaf_a = t.nodes[a].ch[0] < 0 && t.nodes[a].beta, leaf_b = t.nodes[b].ch[0] < 0 && t.nodes[b].beta;
        bool ga = leaf_a || (c.beta && !t.nodes[a].beta && (A & closed).any());
        bool gb = leaf_b || (c.beta && !t.nodes[b].beta && (B & closed).any());
        if (ga && !leaf_a) A = A.andnot(closed) | beta;
        if (gb && !leaf_b) B = B.andnot(closed) | beta;
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
            if (rows_side && tn_tc_narrow(m.count(), nn.count(), k.count())) {
                // a 32-column tensor-core tile: the long side must be the rows
                if (m.count() < nn.count()) { std::swap(a, b); std::swap(m, nn); std::swap(ga, gb); }
            } else if (m_low != rows_side) {
                std::swap(a, b);
                std::swap(m, nn);
                std::swap(ga, gb);
            }
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
        std::vector<int> la, lb;
        la.insert(la.end(), vk.begin(), vk.end());
        la.insert(la.end(), vm.begin(), vm.end());
        la.insert(la.end(), vb.begin(), vb.end());
        lb.insert(lb.end(), vk.begin(), vk.end());
        lb.insert(lb.end(), vn.begin(), vn.end());
        lb.insert(lb.end(), vb.begin(), vb.end());
        // a gathered operand is stored as its read layout without the beta bits, then
        // its closed legs (ascending closed position) as the top bits
        auto store = [&](int o, int x, const std::vector<int> &lv, bool g) -> int {
            if (!g) { t.nodes[x].layout = lv; return TN_OK; }
            std::vector<int> st;
            for (int id : lv)
                if (!beta.has(id)) st.push_back(id);
            const std::vector<int> q =
                (t.nodes[x].ch[0] < 0 && t.nodes[x].beta ? tn_leaf_closed(net, x) : t.nodes[x].idx & closed).list();
            if (q.size() > 32 || net.n_beta > 16) { tn_set_error("compile: gather too wide"); return TN_EUNSUPPORTED; }
            s.gat[o] = 1;
            s.g_nq[o] = (int8_t)q.size();
            for (size_t i = 0; i < q.size(); i++) s.g_q[o][i] = (int16_t)(q[i] - net.closed_base);
            for (int tb = 0; tb < net.n_beta; tb++) {
                int pos = -1;
                for (size_t p = 0; p < lv.size(); p++)
                    if (lv[p] == net.beta_base + tb) pos = (int)p;
                if (pos < 0) { tn_set_error("compile: gathered operand without beta bits"); return TN_EINVAL; }
                s.g_pos_beta[o][tb] = (int8_t)pos;
            }
            s.g_nbits[o] = (int8_t)lv.size();
            st.insert(st.end(), q.begin(), q.end());
            t.nodes[x].layout = st;
            return TN_OK;
        };
        int rc = store(0, a, la, ga);
        if (!rc) rc = store(1, b, lb, gb);
        if (rc) return rc;
        steps.push_back(s);
    }
    std::sort(steps.begin(), steps.end(), [](const Step &x, const Step &y) { return x.c < y.c; });
    return TN_OK;
}

// ------------------------------------------------------------------ whole plan

// Cost-model settings of a plan's networks: tensor-core rate in the split precisions and
// the per-step footprint limit (half the HBM budget, in complex64-sized elements).
void tn_cost_settings(Network &net, const tn_plan_opts &o) {
    net.tc_flop_rate = o.precision != TN_PREC_C64 ? 4e14 : 0;
    const double budget = o.hbm_budget_bytes > 0 ? o.hbm_budget_bytes : 64.0 * (1ull << 30);
    net.mem_limit_elems = budget / 8.0 / 2.0;
    net.job_groups = o.job_groups > 1 ? (double)o.job_groups : 1.0;
    net.anneal_iters = std::max(0, o.anneal_iters);
    net.parallel_greedy = o.parallel_search != 0;
}

int tn_tree_and_compile(Network &net, const tn_plan_opts &o, const int32_t *order, int n_order,
                        const Tree *candidate, Tree &tree, std::vector<Step> &steps, uint64_t *E_used,
                        bool tc_roles) {
    if (order) {
        int rc = tn_tree_from_ssa(net, order, n_order, tree);
        if (rc) return rc;
    } else {
        TreeCost tc;
        tn_search_tree(net, o.order_seed, o.order_trials > 0 ? o.order_trials : 64, tree, tc);
        if (candidate) {
            Tree cand = *candidate;
            tn_recompute_deps(net, cand);
            TreeCost cc = tn_tree_cost(net, cand);
            if (cc.time < tc.time) {
                tree = cand;
                if (cand.q_max >= -1) net.q_max = cand.q_max;
            }
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
    } else if (o.n_auto_sliced > 0 || o.max_log2_tensor > 0) {
        // order the unsliced network, slice it (by time, or down to a tensor size), then
        // re-order with the slices (a size-targeted slicing keeps its tree)
        Network net0;
        int rc = tn_build_amp_network(mg, {}, open, o.log2_batches, net0, closed);
        if (rc) return rc;
        tn_cost_settings(net0, o);
        if (o.max_log2_tensor > 0) {
            net0.mem_limit_elems = 0;
            // no annealing of the unsliced tree here: it lowers the unsliced cost with wider
            // tensors, which the size-targeted slicing then pays for with more sliced legs
            // (on the 40-qubit job 24 instead of 18 legs and 8.5x the work over all slices);
            // the sliced tree is annealed per slice under the cap below
            net0.anneal_iters = 0;
        }
        TreeCost tc0;
        tn_search_tree(net0, o.order_seed, o.order_trials > 0 ? o.order_trials : 64, t0, tc0);
        std::vector<int> picked = o.max_log2_tensor > 0 ? tn_width_slice(net0, t0, o.max_log2_tensor, 62)
                                                        : tn_auto_slice(mg, net0, t0, o.n_auto_sliced);
        for (int id : picked) {
            int seg = net0.idx_seg[id], q = 0;
            while (q + 1 < mg.n && mg.seg_base[q + 1] <= seg) q++;
            I.push_back(tn_edge{q, seg - mg.seg_base[q]});
        }
        have_t0 = true;
    }
    int rc = tn_build_amp_network(mg, I, open, o.log2_batches, net, closed);
    if (rc) return rc;
    tn_cost_settings(net, o);
    if (have_t0 && o.max_log2_tensor > 0) {
        // keep the size-targeted tree: its per-slice tensors are what the slicing bounded
        net.q_max = t0.q_max >= -1 ? t0.q_max : net.q_max;
        tree = t0;
        tn_recompute_deps(net, tree);
        // re-optimise its subtrees for the per-slice cost under the size cap: the search
        // priced the unsliced network, where the sliced legs were not yet sliced (kept
        // only when cheaper with every tensor within the cap)
        {
            net.per_slice = true;
            net.cap_bits = o.max_log2_tensor;
            Tree r;
            if (reconfigured(net, tree, r)) {
                r.q_max = tree.q_max;
                int widest = 0;
                for (const Node &nd : r.nodes) widest = std::max(widest, nd.idx.count());
                if (widest <= o.max_log2_tensor && tn_tree_cost(net, r).time < tn_tree_cost(net, tree).time)
                    tree = r;
            }
            net.per_slice = false;
            net.cap_bits = 0;
            tn_recompute_deps(net, tree);
        }
        // optionally anneal it for the per-slice cost under the size cap (kept only when
        // cheaper with every tensor within the cap)
        if (net.anneal_iters > 0) {
            net.per_slice = true;
            net.cap_bits = o.max_log2_tensor;
            Tree a = tree;
            tn_anneal_tree(net, a, net.anneal_iters, o.order_seed);
            int widest = 0;
            for (const Node &nd : a.nodes) widest = std::max(widest, nd.idx.count());
            if (widest <= o.max_log2_tensor && tn_tree_cost(net, a).time < tn_tree_cost(net, tree).time) tree = a;
            net.per_slice = false;
            net.cap_bits = 0;
            tn_recompute_deps(net, tree);
        }
        uint64_t E = net.n_sliced >= 64 ? ~0ull : ((1ull << net.n_sliced) - 1);
        uint64_t E0 = 0;
        rc = tn_compile(net, tree, E0, steps, o.precision != TN_PREC_C64);
        if (rc == TN_EUNSUPPORTED) {
            E0 = E;
            rc = tn_compile(net, tree, E0, steps, o.precision != TN_PREC_C64);
        }
        if (E_used) *E_used = E0;
        return rc;
    }
    return tn_tree_and_compile(net, o, order, n_order, have_t0 ? &t0 : nullptr, tree, steps, E_used,
                               o.precision != TN_PREC_C64);
}
