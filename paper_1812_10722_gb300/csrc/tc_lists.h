// Host construction of the work lists of the tensor-core far field: groups of G consecutive
// target blocks share one MMA (N = G x 64 targets), so each group walks the union of its
// blocks' lists with a mask per entry of the blocks that own it.  Plain C++ (no CUDA types):
// the test suite compiles this header with the host compiler.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <utility>
#include <vector>

namespace lspr {

struct TcEntry {   // layout of int2
    int box, mask;
};
struct TcItem {    // layout of int4
    int group, begin, end, pad;
};
struct TcRange {   // layout of int4
    int s0, s1, mask, pad;
};

// M2P: per group of G consecutive target blocks, the union of the blocks' box lists sorted by
// box, each box with the mask of the blocks whose list holds it, cut into units of at most seg
// boxes of nearly equal size.  items: [nitems][4] = (block, list begin, list end, -) into list
// (box ids); a block's items cover its list.
inline void tc_group_m2p(int64_t nblocks, int G, int seg, const int *list, const int *items, int64_t nitems,
                         std::vector<TcEntry> &out, std::vector<TcItem> &units) {
    out.clear();
    units.clear();
    const int64_t ngroups = (nblocks + G - 1) / G;
    std::vector<std::vector<TcEntry>> per((size_t)ngroups);
    for (int64_t i = 0; i < nitems; ++i) {
        const int *it = items + 4 * i;
        const int64_t g = it[0] / G;
        const int bit = 1 << (it[0] % G);
        for (int l = it[1]; l < it[2]; ++l) per[g].push_back(TcEntry{list[l], bit});
    }
    for (int64_t g = 0; g < ngroups; ++g) {
        std::vector<TcEntry> &v = per[g];
        if (v.empty()) continue;
        std::sort(v.begin(), v.end(), [](const TcEntry &a, const TcEntry &b) { return a.box < b.box; });
        const int64_t start = (int64_t)out.size();
        for (const TcEntry &e : v) {
            if ((int64_t)out.size() > start && out.back().box == e.box)
                out.back().mask |= e.mask;
            else
                out.push_back(e);
        }
        const int64_t n = (int64_t)out.size() - start, k = (n + seg - 1) / seg;
        for (int64_t q = 0; q < k; ++q)
            units.push_back(TcItem{(int)g, (int)(start + n * q / k), (int)(start + n * (q + 1) / k), 0});
    }
}

// P2P: per group, the blocks' source ranges are cut at every range end (a sweep over the sorted
// ends with one coverage count per block); pieces with the same mask that touch are merged,
// pieces longer than seg_src are split, and consecutive pieces are packed into units of at most
// seg_src sources.  items: [nitems][4] = (block, source begin, source end, -); the ranges of one
// block do not overlap.  Returns the number of sources over all pieces.
inline int64_t tc_group_p2p(int64_t nblocks, int G, int seg_src, const int *items, int64_t nitems,
                            std::vector<TcRange> &out, std::vector<TcItem> &units) {
    out.clear();
    units.clear();
    int64_t total = 0;
    const int64_t ngroups = (nblocks + G - 1) / G;
    std::vector<std::vector<std::pair<int, int>>> ev((size_t)ngroups);   // (position, +-(block + 1))
    for (int64_t i = 0; i < nitems; ++i) {
        const int *it = items + 4 * i;
        if (it[2] <= it[1]) continue;
        const int64_t g = it[0] / G;
        const int k = it[0] % G + 1;
        ev[g].push_back({it[1], k});
        ev[g].push_back({it[2], -k});
    }
    std::vector<int> cov((size_t)G);
    for (int64_t g = 0; g < ngroups; ++g) {
        std::vector<std::pair<int, int>> &e = ev[g];
        if (e.empty()) continue;
        std::sort(e.begin(), e.end(), [](const std::pair<int, int> &a, const std::pair<int, int> &b) {
            return a.first < b.first;
        });
        std::fill(cov.begin(), cov.end(), 0);
        std::vector<TcRange> pieces;
        for (size_t i = 0; i < e.size();) {
            const int pos = e[i].first;
            for (; i < e.size() && e[i].first == pos; ++i) cov[std::abs(e[i].second) - 1] += e[i].second > 0 ? 1 : -1;
            if (i == e.size()) break;
            int mask = 0;
            for (int k = 0; k < G; ++k) mask |= cov[k] > 0 ? 1 << k : 0;
            const int next = e[i].first;
            if (!mask) continue;
            if (!pieces.empty() && pieces.back().s1 == pos && pieces.back().mask == mask)
                pieces.back().s1 = next;
            else
                pieces.push_back(TcRange{pos, next, mask, 0});
        }
        int64_t u0 = (int64_t)out.size(), usrc = 0;
        for (const TcRange &p : pieces)
            for (int s0 = p.s0; s0 < p.s1; s0 += seg_src) {
                const TcRange q{s0, std::min(p.s1, s0 + seg_src), p.mask, 0};
                const int n = q.s1 - q.s0;
                if (usrc > 0 && usrc + n > seg_src) {
                    units.push_back(TcItem{(int)g, (int)u0, (int)out.size(), 0});
                    u0 = (int64_t)out.size();
                    usrc = 0;
                }
                out.push_back(q);
                usrc += n;
                total += n;
            }
        if ((int64_t)out.size() > u0) units.push_back(TcItem{(int)g, (int)u0, (int)out.size(), 0});
    }
    return total;
}

}  // namespace lspr
