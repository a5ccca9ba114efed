// Randomised check of the tensor-core work lists (paper_1812_10722_gb300/csrc/tc_lists.h)
// against brute force: every (box, block) and (source, block) membership of the blocks' own
// lists is present exactly once in the group lists, nothing else is, and the work units
// partition the lists within their size limits.  Prints "ok" and exits 0, else reports the
// first violation and exits 1.
#include <cstdio>
#include <random>
#include <set>
#include <vector>

#include "tc_lists.h"

using namespace lspr;

static int fail(const char *what, int seed) {
    std::printf("case %d: %s\n", seed, what);
    return 1;
}

static int check_m2p(std::mt19937 &rng, int seed) {
    const int G = 4, seg = 1 + (int)(rng() % 7);
    const int64_t nblocks = 1 + rng() % 23, nboxes = 1 + rng() % 60;
    std::vector<std::set<int>> own((size_t)nblocks);
    std::vector<int> list;
    std::vector<int> items;   // (block, begin, end, 0), a block's list in segments of up to 5
    for (int64_t b = 0; b < nblocks; ++b) {
        const int m = (int)(rng() % (nboxes + 1));
        std::vector<int> boxes;
        for (int q = 0; q < m; ++q) {
            const int x = (int)(rng() % nboxes);
            if (own[b].insert(x).second) boxes.push_back(x);   // a box at most once per block
        }
        for (size_t s = 0; s < boxes.size(); s += 5) {
            const int beg = (int)list.size();
            for (size_t q = s; q < boxes.size() && q < s + 5; ++q) list.push_back(boxes[q]);
            items.insert(items.end(), {(int)b, beg, (int)list.size(), 0});
        }
    }
    std::vector<TcEntry> out;
    std::vector<TcItem> units;
    tc_group_m2p(nblocks, G, seg, list.data(), items.data(), (int64_t)items.size() / 4, out, units);
    std::set<std::pair<int, int>> got;   // (box, block)
    std::vector<int> covered(out.size(), 0);
    for (const TcItem &u : units) {
        if (u.end <= u.begin || u.end - u.begin > seg) return fail("m2p unit size", seed);
        for (int l = u.begin; l < u.end; ++l) {
            ++covered[l];
            if (l > u.begin && out[l].box <= out[l - 1].box) return fail("m2p boxes not sorted", seed);
            for (int k = 0; k < G; ++k)
                if (out[l].mask >> k & 1) {
                    const int blk = u.group * G + k;
                    if (blk >= nblocks || !own[blk].count(out[l].box)) return fail("m2p foreign entry", seed);
                    if (!got.insert({out[l].box, blk}).second) return fail("m2p duplicate", seed);
                }
            if (!out[l].mask) return fail("m2p empty mask", seed);
        }
    }
    for (int c : covered)
        if (c != 1) return fail("m2p units do not partition the list", seed);
    size_t want = 0;
    for (auto &s : own) want += s.size();
    if (got.size() != want) return fail("m2p entries missing", seed);
    return 0;
}

static int check_p2p(std::mt19937 &rng, int seed) {
    const int G = 4, seg = 1 + (int)(rng() % 40);
    const int64_t nblocks = 1 + rng() % 23;
    const int nsrc = 1 + (int)(rng() % 300);
    std::vector<std::vector<char>> own((size_t)nblocks, std::vector<char>((size_t)nsrc, 0));
    std::vector<int> items;
    for (int64_t b = 0; b < nblocks; ++b) {
        // disjoint ranges, some adjacent (as the tree's merged and chunked leaf ranges)
        int pos = (int)(rng() % 20);
        while (pos < nsrc) {
            const int len = 1 + (int)(rng() % 30), end = std::min(nsrc, pos + len);
            if (rng() % 3) {
                items.insert(items.end(), {(int)b, pos, end, 0});
                for (int s = pos; s < end; ++s) own[b][s] = 1;
            }
            pos = end + (rng() % 2 ? 0 : (int)(rng() % 15));
        }
    }
    std::vector<TcRange> out;
    std::vector<TcItem> units;
    const int64_t total = tc_group_p2p(nblocks, G, seg, items.data(), (int64_t)items.size() / 4, out, units);
    std::vector<std::vector<char>> got((size_t)nblocks, std::vector<char>((size_t)nsrc, 0));
    std::vector<int> covered(out.size(), 0);
    int64_t sum = 0;
    for (const TcItem &u : units) {
        int64_t n = 0;
        for (int i = u.begin; i < u.end; ++i) {
            ++covered[i];
            const TcRange &r = out[i];
            if (r.s1 <= r.s0 || !r.mask) return fail("p2p empty piece", seed);
            if (i > u.begin && r.s0 < out[i - 1].s1) return fail("p2p pieces overlap or unsorted", seed);
            n += r.s1 - r.s0;
            for (int k = 0; k < G; ++k)
                if (r.mask >> k & 1) {
                    const int blk = u.group * G + k;
                    if (blk >= nblocks) return fail("p2p block past the end", seed);
                    for (int s = r.s0; s < r.s1; ++s) {
                        if (!own[blk][s]) return fail("p2p foreign source", seed);
                        if (got[blk][s]++) return fail("p2p duplicate source", seed);
                    }
                }
        }
        if (n > seg || n == 0) return fail("p2p unit size", seed);
        sum += n;
    }
    for (int c : covered)
        if (c != 1) return fail("p2p units do not partition the pieces", seed);
    if (sum != total) return fail("p2p source count", seed);
    for (int64_t b = 0; b < nblocks; ++b)
        for (int s = 0; s < nsrc; ++s)
            if (own[b][s] != got[b][s]) return fail("p2p source missing", seed);
    return 0;
}

int main() {
    for (int seed = 0; seed < 2000; ++seed) {
        std::mt19937 rng((unsigned)seed);
        if (check_m2p(rng, seed) || check_p2p(rng, seed)) return 1;
    }
    std::printf("ok\n");
    return 0;
}
