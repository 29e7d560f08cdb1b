// lms_host.cpp - host-side logic of liblms: mesh validation, the vertex
// orderings, the first-fit colouring and the reuse-distance profile.  Pure C++,
// no device work; built with -ffp-contract=off (the only floating-point work
// here is comparing keys).
//
// Orderings follow Aupy, Park & Raghavan, "Locality-Aware Laplacian Mesh
// Smoothing": ORI and BFS as compared in Section 5.2.1, a random ordering as in
// Fig. 1a, and the Reuse Distance Reducing ordering of Algorithm 2
// (Section 4.2).  Readings where the paper is silent:
//   RDR  - keys are (vertex quality, id) ascending; the walk's neighbour lists
//          include boundary vertices; l[0] is the worst member of l; vertices no
//          walk reaches are appended in ascending id (Theorem 1 then holds for
//          every vertex, not only the interior ones its proof covers);
//   BFS  - from vertex 0, neighbours in ascending id, restart at the smallest
//          unvisited id;
//   RANDOM - Fisher-Yates, i = n-1 .. 1, j = splitmix64() mod (i+1);
//   RBFS - the BFS visit order read backwards (the reversed breadth-first order
//          Section 2 reports from Munson and Hovland);
//   BRDR - block RDR, a data-parallel variant of Algorithm 2 (not in the paper):
//          Algorithm 2 inside blocks of LMS_BRDR_BLOCK consecutive BFS positions.
//
// The reuse-distance profile follows Section 2.2 and Table 2: the access trace of one sweep
// (each interior vertex in storage order, optionally itself, then its stored row - the pattern of
// Fig. 3), the reuse distance of each access that repeats an element (distinct elements, or
// accesses, in between), and Table 2's quantiles (the k-th smallest, k = ceil(X m) in double,
// clamped to [1, m]).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <deque>
#include <queue>
#include <vector>

#include "lms_internal.h"

namespace lms {

namespace {
thread_local std::string g_detail;

inline int32_t row_len(const int32_t* row_ptr, int32_t v) { return row_ptr[v + 1] - row_ptr[v]; }

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): state advances by the golden gamma, output is
// the state passed through a variant of the MurmurHash3 finaliser.
struct SplitMix64 {
    uint64_t state;
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ULL;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
};

// Strict total order of Algorithm 2's sort keys.
struct KeyLess {
    const double* q;
    bool operator()(int32_t a, int32_t b) const { return q[a] < q[b] || (q[a] == q[b] && a < b); }
};

void order_random(int32_t n, uint64_t seed, int32_t* out) {
    for (int32_t i = 0; i < n; ++i) out[i] = i;
    SplitMix64 g{seed};
    for (int32_t i = n - 1; i > 0; --i) {
        uint64_t j = g.next() % static_cast<uint64_t>(i + 1);
        std::swap(out[i], out[j]);
    }
}

void order_bfs(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* out) {
    std::vector<uint8_t> visited(n, 0);
    std::vector<int32_t> nb;
    int32_t written = 0, read = 0, next_root = 0;
    while (written < n) {
        while (visited[next_root]) ++next_root;
        visited[next_root] = 1;
        out[written++] = next_root;
        while (read < written) {
            const int32_t v = out[read++];
            const int32_t* r0 = col_idx + row_ptr[v];
            const int32_t* r1 = col_idx + row_ptr[v + 1];
            if (!std::is_sorted(r0, r1)) {  // neighbours are visited in ascending id
                nb.assign(r0, r1);
                std::sort(nb.begin(), nb.end());
                r0 = nb.data();
                r1 = nb.data() + nb.size();
            }
            for (const int32_t* it = r0; it != r1; ++it)
                if (!visited[*it]) {
                    visited[*it] = 1;
                    out[written++] = *it;
                }
        }
    }
}

// Threads for `count` items: up to 16 (and the host's), fewer when a thread would get fewer than
// min_per_thread items.
int64_t parts_for(int64_t count, int64_t min_per_thread) {
    const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
    return std::max<int64_t>(1, std::min<int64_t>({16, hw, count / std::max<int64_t>(1, min_per_thread)}));
}

// Runs f(t, nt, lo, hi) for t = 0 .. nt - 1 (nt = parts_for(count, min_per_thread)) over [0, count) cut
// into nt equal parts, part 0 on the calling thread.
template <typename F>
void parallel_parts(int64_t count, int64_t min_per_thread, F&& f) {
    const int64_t nt = parts_for(count, min_per_thread);
    std::vector<std::thread> pool;
    for (int64_t t = 1; t < nt; ++t)
        pool.emplace_back([&f, count, nt, t] { f(t, nt, count * t / nt, count * (t + 1) / nt); });
    f(0, nt, 0, count / nt);
    for (auto& th : pool) th.join();
}

// ids (ascending on entry) in increasing (quality, id): a stable LSD radix sort (16-bit digits) of the
// qualities' bit patterns, which order like the values for non-negative doubles, so equal qualities stay
// in ascending id.  Each pass counts digits per thread part, turns the counts into per-(digit, part)
// offsets and scatters each part in order, which keeps the sort stable.
void sort_by_quality(std::vector<int32_t>& ids, const double* q) {
    const size_t m = ids.size();
    std::vector<uint64_t> key(m), key2(m);
    std::vector<int32_t> ids2(m);
    parallel_parts(int64_t(m), 1 << 16, [&](int64_t, int64_t, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            const double x = q[ids[i]] == 0.0 ? 0.0 : q[ids[i]];  // -0.0 sorts with +0.0
            std::memcpy(&key[i], &x, sizeof(double));
        }
    });
    constexpr size_t kDigits = 65536;
    std::vector<size_t> count;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 16 * pass;
        bool one_digit = true;  // one digit value only: already ordered
        const uint64_t d0 = (key[0] >> shift) & 0xffff;
        for (size_t i = 0; i < m && one_digit; ++i) one_digit = ((key[i] >> shift) & 0xffff) == d0;
        if (one_digit) continue;
        const int64_t parts = parts_for(int64_t(m), 1 << 16);
        count.assign(size_t(parts) * kDigits, 0);
        // count[t * kDigits + d]: keys of part t with digit d, then the offset of the first of them
        parallel_parts(int64_t(m), 1 << 16, [&](int64_t t, int64_t, int64_t lo, int64_t hi) {
            size_t* c = count.data() + size_t(t) * kDigits;
            for (int64_t i = lo; i < hi; ++i) ++c[(key[i] >> shift) & 0xffff];
        });
        size_t at = 0;
        for (size_t d = 0; d < kDigits; ++d)
            for (int64_t t = 0; t < parts; ++t) {
                const size_t c = count[size_t(t) * kDigits + d];
                count[size_t(t) * kDigits + d] = at;
                at += c;
            }
        parallel_parts(int64_t(m), 1 << 16, [&](int64_t t, int64_t, int64_t lo, int64_t hi) {
            size_t* c = count.data() + size_t(t) * kDigits;
            for (int64_t i = lo; i < hi; ++i) {
                const size_t to = c[(key[i] >> shift) & 0xffff]++;
                key2[to] = key[i];
                ids2[to] = ids[i];
            }
        });
        key.swap(key2);
        ids.swap(ids2);
    }
}

// Algorithm 2.  Every vertex gets its rank in increasing (quality, id) order once; the seeds are the
// interior vertices in rank order, and every CSR row is sorted by rank once (in parallel), so the walk's
// list l - the unprocessed neighbours of the current vertex by increasing key - is the current row with
// the processed members skipped.  `done` = processed (the walk has expanded the vertex), `placed` =
// sorted (it has a position in the new order).
void order_rdr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
               const double* q, int32_t* out) {
    std::vector<int32_t> by_key(n);
    for (int32_t v = 0; v < n; ++v) by_key[v] = v;
    bool non_negative = true;
    for (int32_t v = 0; v < n; ++v) non_negative = non_negative && q[v] >= 0.0;
    if (non_negative)
        sort_by_quality(by_key, q);
    else
        std::sort(by_key.begin(), by_key.end(), KeyLess{q});
    std::vector<int32_t> rank(n);
    parallel_parts(n, 1 << 16, [&](int64_t, int64_t, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) rank[by_key[i]] = int32_t(i);
    });
    std::vector<int32_t> row(col_idx, col_idx + row_ptr[n]);
    parallel_parts(n, 1 << 16, [&](int64_t, int64_t, int64_t lo, int64_t hi) {  // rows are short: insertion sort
        for (int64_t v = lo; v < hi; ++v)
            for (int32_t e = row_ptr[v] + 1; e < row_ptr[v + 1]; ++e)
                for (int32_t k = e; k > row_ptr[v] && rank[row[k]] < rank[row[k - 1]]; --k) std::swap(row[k], row[k - 1]);
    });

    // the walk moves between neighbours, so it runs over vertex ids (nearby in memory); the seeds are
    // scanned in rank order over a bitmap by rank of the vertices that are boundary or processed
    constexpr uint8_t kDone = 1, kPlaced = 2;
    std::vector<uint8_t> state(n, 0);
    std::vector<uint64_t> skip((size_t(n) + 63) / 64, 0);
    for (int32_t v = 0; v < n; ++v)
        if (is_boundary[v]) skip[size_t(rank[v]) >> 6] |= uint64_t(1) << (rank[v] & 63);
    int32_t pos = 0;
    auto place = [&](int32_t v) {
        if (!(state[v] & kPlaced)) {
            state[v] |= kPlaced;
            out[pos++] = v;
        }
    };
    auto process = [&](int32_t v) {
        state[v] |= kDone;
        skip[size_t(rank[v]) >> 6] |= uint64_t(1) << (rank[v] & 63);
    };
    for (size_t w = 0; w < skip.size(); ++w) {
        for (uint64_t free = ~skip[w]; free != 0; free = ~skip[w]) {
            const int64_t i = int64_t(w) * 64 + __builtin_ctzll(free);
            if (i >= n) break;
            const int32_t s = by_key[i];  // the worst interior vertex not yet processed
            place(s);
            process(s);
            // the next seed is usually far from this walk: start loading its row now
            for (size_t x = w, k = 0; x < skip.size() && k < 4; ++x, ++k) {
                const uint64_t ahead = ~skip[x] & (x == w ? ~uint64_t(0) << 1 << (i & 63) : ~uint64_t(0));
                if (ahead == 0) continue;
                const int64_t j = int64_t(x) * 64 + __builtin_ctzll(ahead);
                if (j < n) {
                    __builtin_prefetch(row_ptr + by_key[j]);
                    __builtin_prefetch(row.data() + row_ptr[by_key[j]]);
                }
                break;
            }
            for (int32_t cur = s;;) {
                int32_t next = -1;  // l[0]
                for (int32_t e = row_ptr[cur]; e < row_ptr[cur + 1]; ++e) {
                    const int32_t u = row[e];
                    if (state[u] & kDone) continue;
                    if (next < 0) {  // l[0] is known: start loading its row while the rest of l is placed
                        next = u;
                        __builtin_prefetch(row_ptr + u);
                        __builtin_prefetch(row.data() + row_ptr[u]);
                    }
                    place(u);
                }
                if (next < 0) break;
                process(next);
                cur = next;
            }
        }
    }
    for (int32_t v = 0; v < n; ++v) place(v);  // vertices no walk reached, ascending id
}

// Block RDR (a data-parallel variant of Algorithm 2; not in the paper): the BFS order `bfs` cut into
// blocks of `block` consecutive positions, Algorithm 2 run on each block's own subgraph (walks only
// through vertices of the block; members no walk reached follow in ascending id), blocks kept in BFS
// order.  Blocks are independent, so host threads take them in turn.
void order_brdr(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                const double* q, int32_t block, const int32_t* bfs, int32_t* out) {
    KeyLess less{q};
    std::vector<int32_t> blk(n);
    for (int32_t k = 0; k < n; ++k) blk[bfs[k]] = k / block;
    std::vector<uint8_t> done(n, 0), placed(n, 0);
    const int32_t nblocks = (n + block - 1) / block;
    std::atomic<int32_t> next(0);
    auto worker = [&]() {
        std::vector<int32_t> seeds, l, rest;
        for (int32_t j; (j = next++) < nblocks;) {
            const int32_t start = j * block, end = std::min(n, start + block);
            seeds.clear();
            for (int32_t k = start; k < end; ++k)
                if (!is_boundary[bfs[k]]) seeds.push_back(bfs[k]);
            std::sort(seeds.begin(), seeds.end(), less);
            int32_t pos = start;
            auto place = [&](int32_t v) {
                if (!placed[v]) {
                    placed[v] = 1;
                    out[pos++] = v;
                }
            };
            auto gather = [&](int32_t v) {  // unprocessed neighbours inside the block, by increasing key
                l.clear();
                for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                    const int32_t u = col_idx[e];
                    if (blk[u] != j || done[u]) continue;
                    l.push_back(u);
                    for (size_t k = l.size() - 1; k > 0 && less(l[k], l[k - 1]); --k) std::swap(l[k], l[k - 1]);
                }
            };
            for (int32_t sd : seeds) {
                if (done[sd]) continue;
                place(sd);
                done[sd] = 1;
                gather(sd);
                while (!l.empty()) {
                    for (int32_t u : l) place(u);
                    const int32_t w = l.front();
                    done[w] = 1;
                    gather(w);
                }
            }
            rest.clear();
            for (int32_t k = start; k < end; ++k)
                if (!placed[bfs[k]]) rest.push_back(bfs[k]);
            std::sort(rest.begin(), rest.end());
            for (int32_t v : rest) place(v);
        }
    };
    // a thread per 16 blocks at most: small meshes (a batch's) stay on the calling thread
    const unsigned nt = std::max(1u, std::min({16u, std::thread::hardware_concurrency(), unsigned(nblocks / 16)}));
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
}

// Reuse distances of one sweep's access trace.  Distinct-element distances use a Fenwick tree over
// access times holding a 1 at the latest access of every element seen so far: for an access at
// time t to an element last accessed at time p, the elements accessed in between are the marks
// after p, i.e. (elements seen) - prefix(p).
int reuse_profile(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                  const int32_t* new_to_old, int32_t with_vertex, int32_t measure, int32_t nq, const double* q,
                  int64_t* out_q, double* mean, int64_t* n_accesses, int64_t* n_reuses, int64_t* hist) {
    if (n <= 0 || !row_ptr || !is_boundary || (measure != LMS_REUSE_DISTINCT && measure != LMS_REUSE_ACCESSES) ||
        nq < 0 || (nq > 0 && (!q || !out_q)))
        return LMS_ERR_ARG;
    for (int32_t i = 0; i < nq; ++i)
        if (!(q[i] >= 0.0 && q[i] <= 1.0)) return LMS_ERR_ARG;
    if (row_ptr[0] != 0) return LMS_ERR_CSR;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return LMS_ERR_CSR;
    const int32_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return LMS_ERR_ARG;
    for (int32_t e = 0; e < nnz; ++e)
        if (col_idx[e] < 0 || col_idx[e] >= n) return LMS_ERR_CSR;
    if (new_to_old) {
        std::vector<uint8_t> hit(n, 0);
        for (int32_t k = 0; k < n; ++k) {
            const int32_t v = new_to_old[k];
            if (v < 0 || v >= n || hit[v]) return LMS_ERR_ARG;
            hit[v] = 1;
        }
    }
    int64_t len = 0;
    for (int32_t v = 0; v < n; ++v)
        if (!is_boundary[v]) len += row_len(row_ptr, v) + (with_vertex ? 1 : 0);
    if (len >= (int64_t(1) << 32)) return LMS_ERR_ARG;

    std::vector<int64_t> last(n, -1);
    std::vector<uint32_t> dist;
    dist.reserve(size_t(len));
    std::vector<uint32_t> bit;  // Fenwick tree over times 1..len (distinct measure only)
    if (measure == LMS_REUSE_DISTINCT) bit.assign(size_t(len) + 1, 0u);
    int64_t t = 0, seen = 0;
    auto access = [&](int32_t x) {
        const int64_t p = last[x];
        if (p >= 0) {
            uint32_t d;
            if (measure == LMS_REUSE_ACCESSES) {
                d = uint32_t(t - p - 1);
            } else {
                int64_t before = 0;  // marks at times <= p
                for (int64_t i = p + 1; i > 0; i -= i & -i) before += bit[i];
                d = uint32_t(seen - before);
                for (int64_t i = p + 1; i <= len; i += i & -i) --bit[i];
            }
            dist.push_back(d);
        } else {
            ++seen;
        }
        if (measure == LMS_REUSE_DISTINCT)
            for (int64_t i = t + 1; i <= len; i += i & -i) ++bit[i];
        last[x] = t++;
    };
    for (int32_t k = 0; k < n; ++k) {
        const int32_t v = new_to_old ? new_to_old[k] : k;
        if (is_boundary[v]) continue;
        if (with_vertex) access(v);
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) access(col_idx[e]);
    }
    std::vector<uint32_t>().swap(bit);
    const int64_t m = int64_t(dist.size());
    if (n_accesses) *n_accesses = len;
    if (n_reuses) *n_reuses = m;
    if (hist) {  // bucket 0: distance 0; bucket b >= 1: distances in [2^(b-1), 2^b)
        std::fill(hist, hist + 33, 0);
        for (uint32_t d : dist) ++hist[d == 0 ? 0 : 32 - __builtin_clz(d)];
    }
    if (mean) {
        uint64_t sum = 0;
        for (uint32_t d : dist) sum += d;
        *mean = m > 0 ? double(sum) / double(m) : 0.0;
    }
    // quantiles in increasing k: each selection narrows the range of the next
    std::vector<std::pair<int64_t, int32_t>> ks;
    for (int32_t i = 0; i < nq; ++i) {
        int64_t k = int64_t(std::ceil(q[i] * double(m)));
        ks.push_back({std::min(std::max(k, int64_t(1)), std::max(m, int64_t(1))), i});
    }
    std::sort(ks.begin(), ks.end());
    auto lo = dist.begin();
    for (const auto& [k, i] : ks) {
        if (m == 0) {
            out_q[i] = -1;
            continue;
        }
        auto it = dist.begin() + (k - 1);
        if (it >= lo) {
            std::nth_element(lo, it, dist.end());
            lo = it;
        }
        out_q[i] = int64_t(*it);
    }
    return LMS_OK;
}

}  // namespace

void set_error_detail(const std::string& s) { g_detail = s; }
const std::string& error_detail() { return g_detail; }

int validate_mesh(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                  int32_t ntri, const int32_t* tri) {
    if (n <= 0 || !row_ptr || !is_boundary || ntri < 0 || (ntri > 0 && !tri)) return LMS_ERR_ARG;
    if (row_ptr[0] != 0) return LMS_ERR_CSR;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return LMS_ERR_CSR;
    const int32_t nnz = row_ptr[n];
    if (nnz > 0 && !col_idx) return LMS_ERR_ARG;
    for (int32_t e = 0; e < nnz; ++e)
        if (col_idx[e] < 0 || col_idx[e] >= n) return LMS_ERR_CSR;
    // sorted copy of every row: self-loops, duplicates, and symmetry by binary search
    std::vector<int32_t> sorted(col_idx, col_idx + nnz);
    for (int32_t v = 0; v < n; ++v) {
        int32_t* r = sorted.data() + row_ptr[v];
        std::sort(r, r + row_len(row_ptr, v));
        for (int32_t k = 0; k < row_len(row_ptr, v); ++k) {
            if (r[k] == v) return LMS_ERR_CSR;
            if (k > 0 && r[k] == r[k - 1]) return LMS_ERR_CSR;
        }
    }
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t u = sorted[e];
            const int32_t* b = sorted.data() + row_ptr[u];
            if (!std::binary_search(b, b + row_len(row_ptr, u), v)) return LMS_ERR_CSR;
        }
    for (int32_t v = 0; v < n; ++v)
        if (!is_boundary[v] && row_len(row_ptr, v) == 0) return LMS_ERR_ISOLATED;
    for (int64_t t = 0; t < ntri; ++t) {
        int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) return LMS_ERR_ARG;
        if (a == b || b == c || a == c) return LMS_ERR_ARG;
    }
    return LMS_OK;
}

int order_vertices(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const double* q_v, int ordering, uint64_t seed, int32_t* new_to_old) {
    if (n <= 0 || !row_ptr || !new_to_old) return LMS_ERR_ARG;
    switch (ordering) {
        case LMS_ORI:
            for (int32_t i = 0; i < n; ++i) new_to_old[i] = i;
            return LMS_OK;
        case LMS_RANDOM:
            order_random(n, seed, new_to_old);
            return LMS_OK;
        case LMS_BFS:
            if (!col_idx && row_ptr[n] > 0) return LMS_ERR_ARG;
            order_bfs(n, row_ptr, col_idx, new_to_old);
            return LMS_OK;
        case LMS_RDR:
            if (!q_v || !is_boundary || (!col_idx && row_ptr[n] > 0)) return LMS_ERR_ARG;
            order_rdr(n, row_ptr, col_idx, is_boundary, q_v, new_to_old);
            return LMS_OK;
        case LMS_RBFS:
            if (!col_idx && row_ptr[n] > 0) return LMS_ERR_ARG;
            order_bfs(n, row_ptr, col_idx, new_to_old);
            std::reverse(new_to_old, new_to_old + n);
            return LMS_OK;
        case LMS_BRDR: {
            if (!q_v || !is_boundary || (!col_idx && row_ptr[n] > 0)) return LMS_ERR_ARG;
            std::vector<int32_t> bfs(n);
            order_bfs(n, row_ptr, col_idx, bfs.data());
            order_brdr(n, row_ptr, col_idx, is_boundary, q_v, LMS_BRDR_BLOCK, bfs.data(), new_to_old);
            return LMS_OK;
        }
        default:
            return LMS_ERR_ARG;
    }
}

int colour_vertices(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    const int32_t* new_to_old, int32_t* colour, int32_t* ncolours) {
    if (n <= 0 || !row_ptr || !is_boundary || !new_to_old || !colour || !ncolours) return LMS_ERR_ARG;
    std::fill(colour, colour + n, -1);
    std::vector<uint8_t> taken;
    int32_t count = 0;
    for (int32_t k = 0; k < n; ++k) {
        int32_t v = new_to_old[k];
        if (v < 0 || v >= n) return LMS_ERR_ARG;
        if (is_boundary[v]) continue;
        uint64_t mask = 0;  // colours 0..63 of coloured neighbours; larger ones tracked in `taken`
        bool wide = false;
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            int32_t c = colour[col_idx[e]];
            if (c < 0) continue;
            if (c < 64) {
                mask |= 1ULL << c;
            } else {
                if (!wide) {
                    taken.assign(row_len(row_ptr, v) + 1, 0);
                    wide = true;
                }
                if (c - 64 < static_cast<int32_t>(taken.size())) taken[c - 64] = 1;
            }
        }
        int32_t c;
        if (~mask != 0) {
            c = __builtin_ctzll(~mask);
        } else {
            c = 64;
            while (wide && c - 64 < static_cast<int32_t>(taken.size()) && taken[c - 64]) ++c;
        }
        colour[v] = c;
        count = std::max(count, c + 1);
    }
    *ncolours = count;
    return LMS_OK;
}

// Block order of the in-place sweep for a block Gauss-Seidel: tiles of `tile` consecutive storage
// positions, coloured first-fit in ascending tile index so that no two tiles of a colour share an edge
// between interior vertices; interior vertices ordered by (tile colour, tile, vertex colour of the
// first-fit vertex colouring, storage position).  Tiles of one colour, and one colour's vertices inside a
// tile, are independent.  Tile adjacency is gathered per tile and deduplicated with a stamp array;
// the order is two stable counting sorts (tiles by colour, then each tile's vertices by colour).
int block_order(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                const int32_t* new_to_old, int32_t tile, int32_t* tile_colour, int32_t* ntile_colours,
                int32_t* order, int32_t* n_order, int32_t* vertex_colour, int32_t* nvertex_colours) {
    if (n <= 0 || !row_ptr || !col_idx || !is_boundary || !new_to_old || tile < 1 || !tile_colour ||
        !ntile_colours || !order || !n_order)
        return LMS_ERR_ARG;
    std::vector<int32_t> own;
    if (!vertex_colour) own.resize(n);
    int32_t* colour = vertex_colour ? vertex_colour : own.data();
    int32_t nc = 0;
    if (int rc = colour_vertices(n, row_ptr, col_idx, is_boundary, new_to_old, colour, &nc)) return rc;
    if (nvertex_colours) *nvertex_colours = nc;
    std::vector<int32_t> pos(n);
    for (int32_t k = 0; k < n; ++k) pos[new_to_old[k]] = k;
    const int32_t ntiles = static_cast<int32_t>((static_cast<int64_t>(n) + tile - 1) / tile);
    // first-fit tile colours; stamp[c] == t + 1 marks colour c as taken by a neighbour of tile t
    std::vector<int32_t> stamp(static_cast<size_t>(ntiles) + 1, 0);
    int32_t nt = 0;
    for (int32_t t = 0; t < ntiles; ++t) {
        const int32_t k0 = t * tile, k1 = static_cast<int32_t>(std::min<int64_t>(static_cast<int64_t>(k0) + tile, n));
        for (int32_t k = k0; k < k1; ++k) {
            const int32_t v = new_to_old[k];
            if (is_boundary[v]) continue;
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                const int32_t u = col_idx[e];
                if (is_boundary[u]) continue;
                const int32_t tu = pos[u] / tile;
                if (tu < t) stamp[tile_colour[tu]] = t + 1;  // tiles above t are not coloured yet
            }
        }
        int32_t c = 0;
        while (stamp[c] == t + 1) ++c;
        tile_colour[t] = c;
        nt = std::max(nt, c + 1);
    }
    // tiles by colour (stable), then each tile's interior vertices by colour (stable)
    std::vector<int32_t> tile_start(static_cast<size_t>(nt) + 1, 0), tiles(ntiles);
    for (int32_t t = 0; t < ntiles; ++t) ++tile_start[tile_colour[t] + 1];
    for (int32_t c = 0; c < nt; ++c) tile_start[c + 1] += tile_start[c];
    for (int32_t t = 0; t < ntiles; ++t) tiles[tile_start[tile_colour[t]]++] = t;
    std::vector<int32_t> count(static_cast<size_t>(nc) + 1);
    int32_t m = 0;
    for (int32_t t : tiles) {
        const int32_t k0 = t * tile, k1 = static_cast<int32_t>(std::min<int64_t>(static_cast<int64_t>(k0) + tile, n));
        std::fill(count.begin(), count.end(), 0);
        for (int32_t k = k0; k < k1; ++k) {
            const int32_t v = new_to_old[k];
            if (!is_boundary[v]) ++count[colour[v] + 1];
        }
        for (int32_t c = 0; c < nc; ++c) count[c + 1] += count[c];
        for (int32_t k = k0; k < k1; ++k) {
            const int32_t v = new_to_old[k];
            if (!is_boundary[v]) order[m + count[colour[v]]++] = v;
        }
        m += count[nc];
    }
    *ntile_colours = nt;
    *n_order = m;
    return LMS_OK;
}

int block_tables(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                 const int32_t* new_to_old, int32_t tile, BlockTables& out) {
    if (n <= 0 || !new_to_old || tile < 1) return LMS_ERR_ARG;
    const int32_t ntiles = static_cast<int32_t>((static_cast<int64_t>(n) + tile - 1) / tile);
    std::vector<int32_t> tile_colour(ntiles), order(n), colour(n);
    int32_t ntc = 0, m = 0, nc = 0;
    // the vertex colouring block_order computes is the one the colour groups need
    if (int rc = block_order(n, row_ptr, col_idx, is_boundary, new_to_old, tile, tile_colour.data(), &ntc,
                             order.data(), &m, colour.data(), &nc))
        return rc;
    nc = std::max(1, nc);
    std::vector<int32_t> pos(n);
    for (int32_t k = 0; k < n; ++k) pos[new_to_old[k]] = k;
    out.verts.assign(m, 0);
    out.groups.clear();
    std::vector<int32_t> listed_tc;
    int32_t cur_tile = -1;
    for (int32_t i = 0; i < m; ++i) {
        const int32_t v = order[i], t = pos[v] / tile;
        if (t != cur_tile) {  // a listed tile begins: its nc + 1 group offsets start at i
            cur_tile = t;
            listed_tc.push_back(tile_colour[t]);
            out.groups.resize(out.groups.size() + static_cast<size_t>(nc) + 1, i);
        }
        out.verts[i] = pos[v];
        // the tile's vertices come by colour, so group c starts after every vertex of a smaller colour
        const size_t base = out.groups.size() - static_cast<size_t>(nc) - 1;
        for (int32_t c = colour[v] + 1; c <= nc; ++c) out.groups[base + static_cast<size_t>(c)] = i + 1;
    }
    out.tc_ofs.assign(static_cast<size_t>(ntc) + 1, 0);
    for (int32_t tc : listed_tc) ++out.tc_ofs[static_cast<size_t>(tc) + 1];
    for (int32_t c = 0; c < ntc; ++c) out.tc_ofs[static_cast<size_t>(c) + 1] += out.tc_ofs[static_cast<size_t>(c)];
    out.ncolours = nc;
    return LMS_OK;
}

int block_stage_tables(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* new_to_old,
                       int32_t tile, const BlockTables& bt, BlockStageTables& out) {
    if (n <= 0 || !row_ptr || !col_idx || !new_to_old || tile < 1) return LMS_ERR_ARG;
    const int32_t nc = bt.ncolours;
    const size_t listed = bt.groups.size() / (static_cast<size_t>(nc) + 1);
    std::vector<int32_t> pos(n);
    for (int32_t k = 0; k < n; ++k) pos[new_to_old[k]] = k;
    std::vector<int32_t> seen(n, -1), slot(n, 0);  // seen[u] = listed tile that last put u in its halo
    out.tile_info.clear();
    out.halo.clear();
    out.lrow.assign(1, 0);
    out.lcol.clear();
    out.lrow.reserve(bt.verts.size() + 1);
    out.max_slots = 0;
    for (size_t L = 0; L < listed; ++L) {
        const int32_t i0 = bt.groups[L * (nc + 1)], i1 = bt.groups[L * (nc + 1) + nc];
        const int32_t t = bt.verts[i0] / tile;
        const int32_t x = t * tile, y = static_cast<int32_t>(std::min<int64_t>(static_cast<int64_t>(x) + tile, n));
        const int32_t z = static_cast<int32_t>(out.halo.size());
        for (int32_t i = i0; i < i1; ++i) {
            const int32_t v = new_to_old[bt.verts[i]];
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                const int32_t u = pos[col_idx[e]];
                int64_t local;
                if (u >= x && u < y) {
                    local = u - x;
                } else {
                    if (seen[u] != static_cast<int32_t>(L)) {
                        seen[u] = static_cast<int32_t>(L);
                        slot[u] = static_cast<int32_t>(out.halo.size()) - z;
                        out.halo.push_back(u);
                    }
                    local = static_cast<int64_t>(y - x) + slot[u];
                }
                if (local >= 65536) return LMS_ERR_ARG;
                out.lcol.push_back(static_cast<uint16_t>(local));
            }
            out.lrow.push_back(static_cast<int32_t>(out.lcol.size()));
        }
        const int32_t w = static_cast<int32_t>(out.halo.size());
        out.tile_info.insert(out.tile_info.end(), {x, y, z, w});
        out.max_slots = std::max(out.max_slots, (y - x) + (w - z));
        out.max_verts = std::max(out.max_verts, i1 - i0);
        out.max_entries = std::max(out.max_entries, out.lrow[i1] - out.lrow[i0]);
        if (out.max_slots >= 65536) return LMS_ERR_ARG;
    }
    return LMS_OK;
}

}  // namespace lms

extern "C" {

const char* lms_error_string(int status) {
    switch (status) {
        case LMS_OK: return "ok";
        case LMS_ERR_ARG: return "invalid argument (NULL pointer, bad enum, size or index out of range)";
        case LMS_ERR_CSR: return "invalid CSR adjacency (offsets, range, self-loop, duplicate or asymmetry)";
        case LMS_ERR_ISOLATED: return "interior vertex without neighbours";
        case LMS_ERR_NO_TRIANGLES: return "operation needs triangles, none were given";
        case LMS_ERR_CUDA: return "CUDA runtime error";
        case LMS_ERR_OOM: return "out of memory";
        case LMS_ERR_TIMEOUT: return "bounded device-side wait expired";
        case LMS_ERR_STATE: return "call not valid in the current state";
        default: return "unknown status";
    }
}

int lms_validate(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                 int32_t ntri, const int32_t* tri) {
    return lms::validate_mesh(n, row_ptr, col_idx, is_boundary, ntri, tri);
}

int lms_order_host(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const double* q_v, int ordering, uint64_t seed, int32_t* new_to_old) {
    return lms::order_vertices(n, row_ptr, col_idx, is_boundary, q_v, ordering, seed, new_to_old);
}

int lms_color_host(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const int32_t* new_to_old, int32_t* colour, int32_t* ncolours) {
    return lms::colour_vertices(n, row_ptr, col_idx, is_boundary, new_to_old, colour, ncolours);
}

int lms_block_order(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                    const int32_t* new_to_old, int32_t tile, int32_t* tile_colour, int32_t* ntile_colours,
                    int32_t* order, int32_t* n_order) {
    try {
        return lms::block_order(n, row_ptr, col_idx, is_boundary, new_to_old, tile, tile_colour, ntile_colours,
                                order, n_order);
    } catch (const std::bad_alloc&) {
        return LMS_ERR_OOM;
    }
}

int lms_block_walk(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                   const int32_t* new_to_old, int32_t tile, int32_t* seq, int32_t* nseq, int32_t* n_launches) {
    if (!seq || !nseq || !n_launches) return LMS_ERR_ARG;
    try {
        lms::BlockTables bt;
        if (int rc = lms::block_tables(n, row_ptr, col_idx, is_boundary, new_to_old, tile, bt)) return rc;
        // the device sweep's visiting order: one launch per tile colour, block b on listed tile
        // tc_ofs[c] + b, its colour groups in turn (order inside a group and across blocks is free)
        int32_t m = 0, launches = 0;
        for (size_t c = 0; c + 1 < bt.tc_ofs.size(); ++c) {
            if (bt.tc_ofs[c + 1] > bt.tc_ofs[c]) ++launches;
            for (int32_t t = bt.tc_ofs[c]; t < bt.tc_ofs[c + 1]; ++t) {
                const int32_t* g = bt.groups.data() + static_cast<size_t>(t) * (bt.ncolours + 1);
                for (int32_t k = 0; k < bt.ncolours; ++k)
                    for (int32_t i = g[k]; i < g[k + 1]; ++i) seq[m++] = new_to_old[bt.verts[i]];
            }
        }
        *nseq = m;
        *n_launches = launches;
        return LMS_OK;
    } catch (const std::bad_alloc&) {
        return LMS_ERR_OOM;
    }
}

int lms_reuse_profile(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const uint8_t* is_boundary,
                      const int32_t* new_to_old, int32_t with_vertex, int32_t measure, int32_t nq, const double* q,
                      int64_t* out_q, double* mean, int64_t* n_accesses, int64_t* n_reuses, int64_t* hist) {
    try {
        return lms::reuse_profile(n, row_ptr, col_idx, is_boundary, new_to_old, with_vertex, measure, nq, q, out_q,
                                  mean, n_accesses, n_reuses, hist);
    } catch (const std::bad_alloc&) {
        return LMS_ERR_OOM;
    }
}

int lms_partition_meshes(int32_t k, const int32_t* n_vertices, int32_t ranks, int32_t* rank_of, int64_t* load) {
    if (k < 1 || ranks < 1 || !n_vertices || !rank_of) return LMS_ERR_ARG;
    for (int32_t m = 0; m < k; ++m)
        if (n_vertices[m] < 1) return LMS_ERR_ARG;
    std::vector<int32_t> by_size(k);
    for (int32_t m = 0; m < k; ++m) by_size[m] = m;
    std::stable_sort(by_size.begin(), by_size.end(),
                     [&](int32_t a, int32_t b) { return n_vertices[a] > n_vertices[b]; });
    // least-loaded rank first; ties to the lower rank
    using Slot = std::pair<int64_t, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t r = 0; r < ranks; ++r) heap.push({0, r});
    std::vector<int64_t> tot(ranks, 0);
    for (int32_t m : by_size) {
        Slot s = heap.top();
        heap.pop();
        rank_of[m] = s.second;
        s.first += n_vertices[m];
        tot[s.second] = s.first;
        heap.push(s);
    }
    if (load)
        for (int32_t r = 0; r < ranks; ++r) load[r] = tot[r];
    return LMS_OK;
}

}  // extern "C"
