// Versions of every node for a slice set and the arena layout of one execution (host
// only; shared by the engine and a CPU test of its invariants).
//
// The arena is planned in step order: first fit, 256-byte granules, a node released after
// the step that consumes it, a gathered operand after its own step.  Batch-independent
// nodes consumed by batch steps (the stem kept for later batch groups) get a reserved
// prefix instead: batch-dependent tensors are rewritten in every group, so the two never
// share memory.
#pragma once

#include <algorithm>
#include <array>
#include <cstddef>
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "tn_internal.h"

// Sliced legs whose both values appear for every slice of the set (the set is closed
// under flipping them): those legs become layout bits, the others explicit versions.
inline uint64_t explicit_legs(const std::vector<uint64_t> &slices, int nI) {
    std::unordered_map<uint64_t, char> in;
    in.reserve(slices.size() * 2);
    for (uint64_t s : slices) in[s] = 1;
    uint64_t all = nI >= 64 ? ~0ull : ((1ull << nI) - 1);
    uint64_t fr = 0;
    for (int b = 0; b < nI; b++) {
        bool closed = true;
        for (uint64_t s : slices)
            if (!in.count(s ^ (1ull << b))) { closed = false; break; }
        if (closed) fr |= 1ull << b;
    }
    return all & ~fr;
}

struct CallLayout {
    std::vector<std::vector<uint64_t>> vals;             // per node: distinct versions
    std::vector<std::unordered_map<uint64_t, int>> index;
    std::vector<long long> nver;
    std::vector<size_t> off;
    std::vector<std::array<size_t, 2>> goff;  // per step: arena offsets of gathered operands
    size_t arena_bytes = 0;
    double flops = 0, flops_beta = 0;
};

inline void layout_call(const Tree &tree, const std::vector<Step> &steps, uint64_t E, int elem,
                 const std::vector<uint64_t> &slices, CallLayout &L) {
    const auto &nodes = tree.nodes;
    const int NN = (int)nodes.size();
    L.vals.assign(NN, {});
    L.index.assign(NN, {});
    L.nver.assign(NN, 0);
    for (int x = 0; x < NN; x++) {
        const uint64_t D = nodes[x].dep & E;
        for (uint64_t s : slices) {
            uint64_t w = s & D;
            if (L.index[x].emplace(w, (int)L.vals[x].size()).second) L.vals[x].push_back(w);
        }
        L.nver[x] = (long long)L.vals[x].size();
    }
    // arena: first fit, children released after their parent's step; beta-free
    // nodes consumed by beta steps stay alive (reused by later batch groups)
    auto tensor_bytes = [&](int x) {
        return (size_t)L.nver[x] * (size_t(1) << nodes[x].layout.size()) * (size_t)elem;
    };
    struct Blk { size_t off, len; };
    std::vector<Blk> freel;
    size_t top = 0;
    auto alloc = [&](size_t len) {
        len = (len + 255) & ~size_t(255);
        for (size_t i = 0; i < freel.size(); i++)
            if (freel[i].len >= len) {
                size_t o = freel[i].off;
                freel[i].off += len;
                freel[i].len -= len;
                if (!freel[i].len) freel.erase(freel.begin() + i);
                return o;
            }
        size_t o = top;
        top += len;
        return o;
    };
    auto dealloc = [&](size_t off, size_t len) {
        len = (len + 255) & ~size_t(255);
        freel.push_back({off, len});
        std::sort(freel.begin(), freel.end(), [](const Blk &a, const Blk &b) { return a.off < b.off; });
        std::vector<Blk> merged;
        for (auto &b : freel) {
            if (!merged.empty() && merged.back().off + merged.back().len == b.off) merged.back().len += b.len;
            else merged.push_back(b);
        }
        if (!merged.empty() && merged.back().off + merged.back().len == top) { top = merged.back().off; merged.pop_back(); }
        freel.swap(merged);
    };
    // Stem tensors kept for later batch groups (batch-free, consumed by a batch step)
    // get a reserved prefix: batch-dependent tensors are rewritten in every group, so
    // the two must never share memory.
    std::vector<char> keep(NN, 0);
    for (const Step &s : steps)
        for (int ch : {s.a, s.b})
            if (nodes[ch].ch[0] >= 0 && !nodes[ch].beta && nodes[s.c].beta) keep[ch] = 1;
    size_t reserved = 0;
    L.off.assign(NN, 0);
    for (const Step &s : steps)
        if (keep[s.c]) {
            L.off[s.c] = reserved;
            reserved += (tensor_bytes(s.c) + 255) & ~size_t(255);
        }
    size_t peak = 0;
    L.flops = L.flops_beta = 0;
    L.goff.assign(steps.size(), {0, 0});
    auto nver_of = [&](int x) -> long long {
        if (nodes[x].ch[0] >= 0) return L.nver[x];
        return 1LL << __builtin_popcountll(nodes[x].dep & E);  // leaf codes
    };
    for (size_t i = 0; i < steps.size(); i++) {
        const Step &s = steps[i];
        // gathered operands live for the step only
        size_t gbytes[2] = {0, 0};
        for (int o = 0; o < 2; o++)
            if (s.gat[o]) {
                gbytes[o] = (size_t)nver_of(o ? s.b : s.a) * (size_t(1) << s.g_nbits[o]) * (size_t)elem;
                L.goff[i][o] = reserved + alloc(gbytes[o]);
            }
        if (!keep[s.c]) L.off[s.c] = reserved + alloc(tensor_bytes(s.c));
        peak = std::max(peak, top);
        for (int o = 0; o < 2; o++)
            if (s.gat[o]) dealloc(L.goff[i][o] - reserved, gbytes[o]);
        for (int ch : {s.a, s.b})
            if (nodes[ch].ch[0] >= 0 && !keep[ch]) dealloc(L.off[ch] - reserved, tensor_bytes(ch));
        const double fl = s.flops_per_version * (double)L.nver[s.c];
        L.flops += fl;
        if (nodes[s.c].beta) L.flops_beta += fl;
    }
    L.arena_bytes = std::max<size_t>(reserved + peak, 256);
}
