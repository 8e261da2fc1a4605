/*
 * CPU oracle for rule-based blocking — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load this library.  The GPU library never links or calls it, and it
 * shares no code, header or table with the GPU library.
 *
 * What it computes is the plain definition of blocking with matching
 * dependencies (Section 2, "Rules", "Semantics" and "Blocking"):
 *
 *   Ca = { (t1, t2) : some MD phi = X -> t.eid = s.eid in Delta has
 *                     h(t1, t2) |= p for every predicate p in X }
 *
 * for a self-join (pairs i < j of one relation) or for two relations R x S
 * (all pairs (i in R, j in S)).  The naive evaluation of Section 4 ("a naive
 * approach ... evaluate each MD in Delta for all pairs") is or_block_literal;
 * or_block_hash only restricts which pairs are looked at, using the fact that
 * a pair can satisfy a precondition only if it agrees on all of its equality
 * predicates, and then evaluates the whole disjunction for each such pair.
 *
 * Predicate semantics (readings where the paper is silent):
 *   - a missing operand makes every predicate false (Example 3: (t2, t3) fails
 *     price equality because t2.price is missing);
 *   - eq        : byte equality of strings, value equality of int32;
 *   - eq_prefix : equality of the first min(k, len) bytes of two strings;
 *   - ed        : unit-cost Levenshtein distance over bytes <= k
 *                 (edit distance of Example 2), by the Wagner-Fischer DP;
 *   - jaccard   : set of all contiguous q-byte substrings (no padding, strings
 *                 shorter than q give the empty set); |A^B| * den >= num * |AuB|
 *                 in integers (Jaccard measure of Example 2);
 *   - absdiff   : fabsf(a - b) <= delta in IEEE binary32, round to nearest even,
 *                 no contraction (compile with -ffp-contract=off).
 *
 * Parity status: ed, jaccard, absdiff, eq and eq_prefix are pinned by the
 * tests (textbook DP properties, brute force, hand-computed cases and the
 * paper's Table 1 / Examples 3 and "(t1, t5)").
 */
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

struct or_col {
    int32_t type;            /* 0 string, 1 int32, 2 fp32 */
    int32_t pad;
    const void *data;        /* string bytes, int32 values or float values */
    const uint32_t *off;     /* strings: n+1 byte offsets */
    const uint8_t *valid;    /* one byte per row, nonzero = present; NULL = all present */
};

struct or_pred {
    int32_t kind;            /* 0 eq, 1 eq_prefix, 2 ed, 3 jaccard, 4 absdiff, 5 const_eq, 6 contain,
                                7 token jaccard */
    int32_t col_t, col_s;    /* column of the left tuple (R) and of the right tuple (S) */
    int32_t k;               /* ed: max distance; eq_prefix: prefix length */
    int32_t q;               /* jaccard, contain: gram length */
    uint32_t num, den;       /* jaccard, contain, token jaccard: threshold num/den */
    float delta;             /* absdiff */
    int32_t side;            /* const_eq: 0 = t.A = c, 1 = s.A = c; contain: whose set divides, 0 = t, 1 = s */
    uint32_t value_len;      /* const_eq: constant bytes (string column) or 4 (int32 column) */
    const void *value;       /* const_eq: the constant */
};

struct Rel {
    int64_t n;
    int ncols;
    const or_col *cols;
};

bool present(const or_col &c, int64_t i) { return c.valid == nullptr || c.valid[i] != 0; }

std::string bytes_of(const or_col &c, int64_t i) {
    const uint8_t *p = static_cast<const uint8_t *>(c.data);
    return std::string(reinterpret_cast<const char *>(p + c.off[i]), c.off[i + 1] - c.off[i]);
}

/* Wagner-Fischer dynamic programme for the Levenshtein distance. */
int64_t levenshtein(const std::string &a, const std::string &b) {
    const size_t m = a.size(), n = b.size();
    std::vector<int64_t> prev(n + 1), cur(n + 1);
    for (size_t j = 0; j <= n; j++) prev[j] = (int64_t)j;
    for (size_t i = 1; i <= m; i++) {
        cur[0] = (int64_t)i;
        for (size_t j = 1; j <= n; j++) {
            int64_t sub = prev[j - 1] + (a[i - 1] == b[j - 1] ? 0 : 1);
            int64_t del = prev[j] + 1;
            int64_t ins = cur[j - 1] + 1;
            cur[j] = std::min(sub, std::min(del, ins));
        }
        std::swap(prev, cur);
    }
    return prev[n];
}

std::set<std::string> qgrams(const std::string &s, int q) {
    std::set<std::string> g;
    if (q <= 0) return g;
    for (size_t i = 0; i + (size_t)q <= s.size(); i++) g.insert(s.substr(i, (size_t)q));
    return g;
}

/* word tokens: the maximal runs of bytes other than the space byte 0x20 */
std::set<std::string> tokens(const std::string &s) {
    std::set<std::string> t;
    size_t i = 0;
    while (i < s.size()) {
        while (i < s.size() && s[i] == ' ') i++;
        size_t j = i;
        while (j < s.size() && s[j] != ' ') j++;
        if (j > i) t.insert(s.substr(i, j - i));
        i = j;
    }
    return t;
}

/* |A n B| * den >= num * |A u B| for two sets */
bool set_jaccard_ge(const std::set<std::string> &A, const std::set<std::string> &B, uint32_t num, uint32_t den) {
    std::vector<std::string> inter;
    std::set_intersection(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(inter));
    uint64_t I = inter.size();
    uint64_t U = A.size() + B.size() - I;
    return I * (uint64_t)den >= (uint64_t)num * U;
}

/* containment of D in the other set E: |D n E| * den >= num * |D| */
bool contain_ge(const std::set<std::string> &D, const std::set<std::string> &E, uint32_t num, uint32_t den) {
    std::vector<std::string> inter;
    std::set_intersection(D.begin(), D.end(), E.begin(), E.end(), std::back_inserter(inter));
    return (uint64_t)inter.size() * (uint64_t)den >= (uint64_t)num * (uint64_t)D.size();
}

bool jaccard_ge(const std::string &a, const std::string &b, int q, uint32_t num, uint32_t den) {
    std::set<std::string> A = qgrams(a, q), B = qgrams(b, q);
    std::vector<std::string> inter;
    std::set_intersection(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(inter));
    uint64_t I = inter.size();
    uint64_t U = A.size() + B.size() - I;
    return I * (uint64_t)den >= (uint64_t)num * U;
}

bool holds(const or_pred &p, const Rel &R, int64_t i, const Rel &S, int64_t j) {
    if (p.kind == 5) {   /* t.A = c (side 0: the left tuple) or s.A = c (side 1: the right tuple) */
        const or_col &c = p.side == 0 ? R.cols[p.col_t] : S.cols[p.col_s];
        const int64_t r = p.side == 0 ? i : j;
        if (!present(c, r)) return false;
        if (c.type == 1) {
            int32_t want;
            std::memcpy(&want, p.value, 4);
            return static_cast<const int32_t *>(c.data)[r] == want;
        }
        return bytes_of(c, r) == std::string(static_cast<const char *>(p.value), p.value_len);
    }
    const or_col &a = R.cols[p.col_t];
    const or_col &b = S.cols[p.col_s];
    if (!present(a, i) || !present(b, j)) return false;
    switch (p.kind) {
    case 0:
        if (a.type == 0 && b.type == 0) return bytes_of(a, i) == bytes_of(b, j);
        if (a.type == 1 && b.type == 1)
            return static_cast<const int32_t *>(a.data)[i] == static_cast<const int32_t *>(b.data)[j];
        return false;
    case 1: {
        std::string x = bytes_of(a, i), y = bytes_of(b, j);
        size_t k = (size_t)std::max(p.k, 0);
        return x.substr(0, std::min(k, x.size())) == y.substr(0, std::min(k, y.size()));
    }
    case 2:
        return levenshtein(bytes_of(a, i), bytes_of(b, j)) <= (int64_t)p.k;
    case 3:
        return jaccard_ge(bytes_of(a, i), bytes_of(b, j), p.q, p.num, p.den);
    case 4: {
        float x = static_cast<const float *>(a.data)[i];
        float y = static_cast<const float *>(b.data)[j];
        volatile float d = x - y;
        return std::fabs((float)d) <= p.delta;
    }
    case 6: {
        std::set<std::string> A = qgrams(bytes_of(a, i), p.q), B = qgrams(bytes_of(b, j), p.q);
        return p.side == 0 ? contain_ge(A, B, p.num, p.den) : contain_ge(B, A, p.num, p.den);
    }
    case 7:
        return set_jaccard_ge(tokens(bytes_of(a, i)), tokens(bytes_of(b, j)), p.num, p.den);
    }
    return false;
}

/* the precondition of one MD: every predicate holds (short-circuit AND) */
bool md_holds(const or_pred *preds, int32_t lo, int32_t hi, const Rel &R, int64_t i, const Rel &S, int64_t j) {
    for (int32_t k = lo; k < hi; k++)
        if (!holds(preds[k], R, i, S, j)) return false;
    return true;
}

/* the disjunction over all MDs: some MD is a witness (short-circuit OR) */
bool dnf_holds(int n_md, const int32_t *md_start, const or_pred *preds, const Rel &R, int64_t i, const Rel &S,
               int64_t j) {
    for (int m = 0; m < n_md; m++)
        if (md_holds(preds, md_start[m], md_start[m + 1], R, i, S, j)) return true;
    return false;
}

/* A self-join reports the unordered pair {i, j} when some MD is a witness at
 * (t_i, t_j) or at (t_j, t_i); with symmetric predicates only the two
 * valuations agree, so the second is evaluated only when some predicate is
 * asymmetric (asym).  R x S pairs have one valuation, (r_i, s_j). */
bool pair_holds(int n_md, const int32_t *md_start, const or_pred *preds, const Rel &R, int64_t i, const Rel &S,
                int64_t j, bool self, bool asym) {
    if (dnf_holds(n_md, md_start, preds, R, i, S, j)) return true;
    return self && asym && dnf_holds(n_md, md_start, preds, R, j, S, i);
}

bool is_equality(const or_pred &p) { return p.kind == 0 || p.kind == 1; }

/* A predicate whose verdict can change when the two tuples swap roles: a
 * constant on one of them, containment, or two different columns. */
bool asymmetric(const or_pred &p) { return p.kind == 5 || p.kind == 6 || p.col_t != p.col_s; }

bool any_asymmetric(int n_md, const int32_t *md_start, const or_pred *preds) {
    for (int32_t k = 0; k < md_start[n_md]; k++)
        if (asymmetric(preds[k])) return true;
    return false;
}

/* The equality predicates a group is keyed on: in a self-join, those that
 * compare a column with itself (t.A = s.B with A != B relates two different
 * columns of the pair's tuples and is checked per pair instead). */
bool groups_on(const or_pred &p, bool self) { return is_equality(p) && (!self || p.col_t == p.col_s); }

/* the grouping key of tuple i for the equality predicates of one MD; false if a value is missing */
bool group_key(const or_pred *preds, int32_t lo, int32_t hi, const Rel &T, int64_t i, bool left, std::string &key,
               bool self) {
    key.clear();
    for (int32_t k = lo; k < hi; k++) {
        const or_pred &p = preds[k];
        if (!groups_on(p, self)) continue;
        const or_col &c = T.cols[left ? p.col_t : p.col_s];
        if (!present(c, i)) return false;
        std::string part;
        if (c.type == 1) {
            int32_t v = static_cast<const int32_t *>(c.data)[i];
            part.assign(reinterpret_cast<const char *>(&v), 4);
        } else {
            part = bytes_of(c, i);
            if (p.kind == 1) part = part.substr(0, std::min((size_t)std::max(p.k, 0), part.size()));
        }
        uint64_t len = part.size();
        key.append(reinterpret_cast<const char *>(&len), 8);
        key.append(part);
    }
    return true;
}

int64_t emit(const std::vector<uint64_t> &v, uint64_t *out, int64_t cap) {
    int64_t n = (int64_t)v.size();
    if (out) std::memcpy(out, v.data(), sizeof(uint64_t) * (size_t)std::min(n, cap));
    return n;
}

}  // namespace

namespace {

struct GramSets { int side, col, q; std::vector<std::vector<std::string>> rows; };

void group_ids(const or_pred *preds, int32_t lo, int32_t hi, const Rel &R, const Rel *S,
               std::vector<int64_t> &gr, std::vector<int64_t> &gs, std::vector<std::vector<int64_t>> &left,
               std::vector<std::vector<int64_t>> &right) {
    bool has_eq = false;
    for (int32_t k = lo; k < hi; k++) has_eq = has_eq || groups_on(preds[k], S == nullptr);
    gr.assign((size_t)R.n, -1);
    if (S) gs.assign((size_t)S->n, -2);
    left.clear();
    right.clear();
    if (!has_eq) {
        left.emplace_back();
        for (int64_t i = 0; i < R.n; i++) { gr[(size_t)i] = 0; left[0].push_back(i); }
        if (S) {
            right.emplace_back();
            for (int64_t j = 0; j < S->n; j++) { gs[(size_t)j] = 0; right[0].push_back(j); }
        }
        return;
    }
    std::unordered_map<std::string, int64_t> index;
    std::string key;
    for (int64_t i = 0; i < R.n; i++) {
        if (!group_key(preds, lo, hi, R, i, true, key, S == nullptr)) continue;
        auto it = index.find(key);
        if (it == index.end()) {
            it = index.emplace(key, (int64_t)left.size()).first;
            left.emplace_back();
        }
        gr[(size_t)i] = it->second;
        left[(size_t)it->second].push_back(i);
    }
    if (!S) return;
    right.resize(left.size());
    for (int64_t j = 0; j < S->n; j++) {
        if (!group_key(preds, lo, hi, *S, j, false, key, false)) { gs[(size_t)j] = -1; continue; }
        auto it = index.find(key);
        if (it == index.end()) continue;
        gs[(size_t)j] = it->second;
        right[(size_t)it->second].push_back(j);
    }
}

/* the q-gram set of every row of one string column, as sorted unique substrings */
void gram_rows(const Rel &T, int col, int q, int n_threads, std::vector<std::vector<std::string>> &rows) {
    rows.assign((size_t)T.n, {});
    const or_col &c = T.cols[col];
    std::atomic<int64_t> next{0};
    auto work = [&]() {
        for (;;) {
            int64_t i0 = next.fetch_add(4096);
            if (i0 >= T.n) break;
            for (int64_t i = i0; i < std::min(T.n, i0 + 4096); i++) {
                if (!present(c, i)) continue;
                std::set<std::string> g = qgrams(bytes_of(c, i), q);
                rows[(size_t)i].assign(g.begin(), g.end());
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < std::max(n_threads, 1); t++) th.emplace_back(work);
    work();
    for (auto &x : th) x.join();
}

/* |A n B| of two sorted unique lists */
uint64_t common(const std::vector<std::string> &A, const std::vector<std::string> &B) {
    size_t a = 0, b = 0;
    uint64_t I = 0;
    while (a < A.size() && b < B.size()) {
        if (A[a] < B[b]) a++;
        else if (B[b] < A[a]) b++;
        else { I++; a++; b++; }
    }
    return I;
}

struct Owned {
    int n_md;
    const int32_t *md_start;
    const or_pred *preds;
    const Rel &R, &S;
    const std::vector<GramSets> &grams;
    bool self;

    const std::vector<std::vector<std::string>> *gram_of(int side, int col, int q) const {
        if (self) side = 0;   /* a self-join reads both tuples from R */
        for (const GramSets &g : grams)
            if (g.side == side && g.col == col && g.q == q) return &g.rows;
        return nullptr;
    }

    bool holds_p(const or_pred &p, int64_t i, int64_t j) const {
        if (p.kind != 3) return holds(p, R, i, S, j);
        if (!present(R.cols[p.col_t], i) || !present(S.cols[p.col_s], j)) return false;
        const auto *A = gram_of(0, p.col_t, p.q), *B = gram_of(1, p.col_s, p.q);
        if (!A || !B) return holds(p, R, i, S, j);
        const std::vector<std::string> &a = (*A)[(size_t)i], &b = (*B)[(size_t)j];
        const uint64_t I = common(a, b), U = a.size() + b.size() - I;
        return I * (uint64_t)p.den >= (uint64_t)p.num * U;
    }

    bool dnf1(int64_t i, int64_t j) const {
        for (int m = 0; m < n_md; m++) {
            bool all = true;
            for (int32_t k = md_start[m]; k < md_start[m + 1] && all; k++) all = holds_p(preds[k], i, j);
            if (all) return true;
        }
        return false;
    }

    /* as pair_holds: both valuations of a self-join pair when a predicate is asymmetric */
    bool dnf(int64_t i, int64_t j) const { return dnf1(i, j) || (self && asym && dnf1(j, i)); }
    bool asym = false;
};

}  // namespace

extern "C" {

int64_t or_edit_distance(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb) {
    return levenshtein(std::string(reinterpret_cast<const char *>(a), (size_t)la),
                       std::string(reinterpret_cast<const char *>(b), (size_t)lb));
}

/* sizes of the q-gram sets and of their intersection */
void or_qgram_sets(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb, int32_t q, int64_t *na, int64_t *nb,
                   int64_t *ni) {
    std::set<std::string> A = qgrams(std::string(reinterpret_cast<const char *>(a), (size_t)la), q);
    std::set<std::string> B = qgrams(std::string(reinterpret_cast<const char *>(b), (size_t)lb), q);
    std::vector<std::string> inter;
    std::set_intersection(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(inter));
    *na = (int64_t)A.size();
    *nb = (int64_t)B.size();
    *ni = (int64_t)inter.size();
}

int32_t or_jaccard_ge(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb, int32_t q, uint32_t num,
                      uint32_t den) {
    return jaccard_ge(std::string(reinterpret_cast<const char *>(a), (size_t)la),
                      std::string(reinterpret_cast<const char *>(b), (size_t)lb), q, num, den) ? 1 : 0;
}

int32_t or_absdiff_le(float a, float b, float delta) {
    volatile float d = a - b;
    return std::fabs((float)d) <= delta ? 1 : 0;
}

/*
 * Naive nested loop (Section 4, first paragraph).  S == NULL means self-join
 * (pairs i < j of R).  Pairs are packed as (i << 32) | j, ascending.
 * Returns the number of pairs; writes at most cap of them.
 */
int64_t or_block_literal(int64_t nR, int32_t ncR, const or_col *R, int64_t nS, int32_t ncS, const or_col *S,
                         int32_t n_md, const int32_t *md_start, const or_pred *preds, uint64_t *out, int64_t cap) {
    Rel r{nR, ncR, R};
    Rel s = S ? Rel{nS, ncS, S} : r;
    std::vector<uint64_t> res;
    for (int64_t i = 0; i < r.n; i++)
        for (int64_t j = S ? 0 : i + 1; j < s.n; j++)
            if (dnf_holds(n_md, md_start, preds, r, i, s, j) || (!S && dnf_holds(n_md, md_start, preds, r, j, s, i)))
                res.push_back(((uint64_t)i << 32) | (uint64_t)j);
    return emit(res, out, cap);
}

/*
 * Same result as or_block_literal, looking only at pairs that agree on all
 * equality predicates of some MD (MDs without one contribute every pair).
 * Also returns, in *n_candidates, the number of distinct such pairs.
 */
int64_t or_block_hash(int64_t nR, int32_t ncR, const or_col *R, int64_t nS, int32_t ncS, const or_col *S,
                      int32_t n_md, const int32_t *md_start, const or_pred *preds, int32_t n_threads, uint64_t *out,
                      int64_t cap, int64_t *n_candidates, int32_t count_candidates) {
    Rel r{nR, ncR, R};
    Rel s = S ? Rel{nS, ncS, S} : r;
    const bool self = (S == nullptr);
    const bool asym = any_asymmetric(n_md, md_start, preds);
    struct Group { std::vector<int64_t> left, right; };
    std::vector<Group> groups;
    for (int m = 0; m < n_md; m++) {
        std::unordered_map<std::string, size_t> index;
        std::string key;
        size_t first = groups.size();
        for (int64_t i = 0; i < r.n; i++) {
            if (!group_key(preds, md_start[m], md_start[m + 1], r, i, true, key, self)) continue;
            auto it = index.find(key);
            if (it == index.end()) { it = index.emplace(key, groups.size()).first; groups.emplace_back(); }
            groups[it->second].left.push_back(i);
        }
        if (!self) {
            for (int64_t j = 0; j < s.n; j++) {
                if (!group_key(preds, md_start[m], md_start[m + 1], s, j, false, key, false)) continue;
                auto it = index.find(key);
                if (it == index.end()) continue;
                groups[it->second].right.push_back(j);
            }
        }
        (void)first;
    }
    std::atomic<size_t> next{0};
    std::vector<std::vector<uint64_t>> res((size_t)std::max(n_threads, 1)), cand((size_t)std::max(n_threads, 1));
    auto work = [&](int t) {
        for (;;) {
            size_t g = next.fetch_add(1);
            if (g >= groups.size()) break;
            const Group &G = groups[g];
            if (self) {
                for (size_t a = 0; a < G.left.size(); a++)
                    for (size_t b = a + 1; b < G.left.size(); b++) {
                        int64_t i = G.left[a], j = G.left[b];
                        uint64_t key = ((uint64_t)i << 32) | (uint64_t)j;
                        if (count_candidates) cand[t].push_back(key);
                        if (pair_holds(n_md, md_start, preds, r, i, s, j, self, asym)) res[t].push_back(key);
                    }
            } else {
                for (int64_t i : G.left)
                    for (int64_t j : G.right) {
                        uint64_t key = ((uint64_t)i << 32) | (uint64_t)j;
                        if (count_candidates) cand[t].push_back(key);
                        if (pair_holds(n_md, md_start, preds, r, i, s, j, self, asym)) res[t].push_back(key);
                    }
            }
        }
    };
    std::vector<std::thread> th;
    int nt = std::max(n_threads, 1);
    for (int t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
    std::vector<uint64_t> all;
    for (auto &v : res) { all.insert(all.end(), v.begin(), v.end()); std::vector<uint64_t>().swap(v); }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    if (n_candidates) {
        if (count_candidates) {
            std::vector<uint64_t> c;
            for (auto &v : cand) { c.insert(c.end(), v.begin(), v.end()); std::vector<uint64_t>().swap(v); }
            std::sort(c.begin(), c.end());
            c.erase(std::unique(c.begin(), c.end()), c.end());
            *n_candidates = (int64_t)c.size();
        } else {
            *n_candidates = -1;
        }
    }
    return emit(all, out, cap);
}

/*
 * Same result as or_block_hash, for relations too large for it (the
 * benchmark's full sizes), in two plain steps:
 *
 *  1. every tuple gets, per MD, the id of its group of equal values of that
 *     MD's equality predicates (-1 when one of them is missing; an MD without
 *     equality predicates puts every tuple in group 0; an S tuple whose values
 *     no R tuple holds gets -2);
 *  2. a pair that agrees on some MD's equality predicates is looked at once,
 *     in the group of the lowest-numbered such MD (two tuples agree on MD m'
 *     iff their group ids of m' are equal and not negative), counted as a
 *     candidate, and the whole disjunction is evaluated for it.
 *
 * Large groups are cut into ranges of their first tuple so that all threads
 * stay busy.  The q-gram set of each string a Jaccard predicate reads is
 * built once per row (the same set of substrings as qgrams(), kept sorted),
 * because the full sizes evaluate it billions of times.  evaluate = 0 only
 * counts the candidates (out may then be NULL).
 */
int64_t or_block_owned(int64_t nR, int32_t ncR, const or_col *R, int64_t nS, int32_t ncS, const or_col *S,
                       int32_t n_md, const int32_t *md_start, const or_pred *preds, int32_t n_threads,
                       int32_t evaluate, uint64_t *out, int64_t cap, int64_t *n_candidates) {
    Rel r{nR, ncR, R};
    Rel s = S ? Rel{nS, ncS, S} : r;
    const bool self = (S == nullptr);
    const int nt = std::max(n_threads, 1);
    // 1. group ids per MD
    std::vector<std::vector<int64_t>> gid_r((size_t)n_md), gid_s((size_t)n_md);
    std::vector<std::vector<std::vector<int64_t>>> left((size_t)n_md), right((size_t)n_md);
    for (int m = 0; m < n_md; m++)
        group_ids(preds, md_start[m], md_start[m + 1], r, self ? nullptr : &s, gid_r[(size_t)m], gid_s[(size_t)m],
                  left[(size_t)m], right[(size_t)m]);
    const std::vector<std::vector<int64_t>> &gid_c = self ? gid_r : gid_s;
    // q-gram sets of the string columns Jaccard predicates read
    std::vector<GramSets> grams;
    if (evaluate) {
        for (int32_t k = 0; k < md_start[n_md]; k++) {
            const or_pred &p = preds[k];
            if (p.kind != 3) continue;
            for (int side = 0; side < (self ? 1 : 2); side++) {
                const int col = side == 0 ? p.col_t : p.col_s;
                bool have = false;
                for (const GramSets &g : grams) have = have || (g.side == side && g.col == col && g.q == p.q);
                if (have) continue;
                grams.push_back(GramSets{side, col, p.q, {}});
                gram_rows(side == 0 ? r : s, col, p.q, nt, grams.back().rows);
            }
        }
    }
    // 2. work units: (MD, group, range of the first tuple's position) of at most ~2^21 pairs
    struct Unit { int m; int64_t g, a0, a1; };
    std::vector<Unit> units;
    for (int m = 0; m < n_md; m++) {
        for (size_t g = 0; g < left[(size_t)m].size(); g++) {
            const int64_t nl = (int64_t)left[(size_t)m][g].size();
            const int64_t nrt = self ? nl : (int64_t)right[(size_t)m][g].size();
            if (nl == 0 || nrt == 0 || (self && nl < 2)) continue;
            int64_t a = 0;
            while (a < nl) {
                int64_t b = a, pairs = 0;
                while (b < nl && pairs < (1 << 21)) { pairs += self ? (nl - 1 - b) : nrt; b++; }
                units.push_back(Unit{m, (int64_t)g, a, b});
                a = b;
            }
        }
    }
    Owned ev{n_md, md_start, preds, r, s, grams, self};
    ev.asym = any_asymmetric(n_md, md_start, preds);
    std::atomic<size_t> next{0};
    std::vector<std::vector<uint64_t>> res((size_t)nt);
    std::vector<int64_t> cand((size_t)nt, 0);
    auto owner_is = [&](int m, int64_t i, int64_t j) {
        for (int mm = 0; mm < m; mm++) {
            const int64_t x = gid_r[(size_t)mm][(size_t)i];
            if (x >= 0 && x == gid_c[(size_t)mm][(size_t)j]) return false;
        }
        return true;
    };
    auto work = [&](int t) {
        for (;;) {
            const size_t u = next.fetch_add(1);
            if (u >= units.size()) break;
            const Unit &U = units[u];
            const std::vector<int64_t> &L = left[(size_t)U.m][(size_t)U.g];
            const std::vector<int64_t> &Rt = self ? L : right[(size_t)U.m][(size_t)U.g];
            for (int64_t a = U.a0; a < U.a1; a++) {
                for (int64_t b = self ? a + 1 : 0; b < (int64_t)Rt.size(); b++) {
                    int64_t i = L[(size_t)a], j = Rt[(size_t)b];
                    if (self && i > j) std::swap(i, j);
                    if (!owner_is(U.m, i, j)) continue;
                    cand[(size_t)t]++;
                    if (evaluate && ev.dnf(i, j)) res[(size_t)t].push_back(((uint64_t)i << 32) | (uint64_t)j);
                }
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
    std::vector<uint64_t> all;
    int64_t c = 0;
    for (int t = 0; t < nt; t++) {
        c += cand[(size_t)t];
        all.insert(all.end(), res[(size_t)t].begin(), res[(size_t)t].end());
    }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    if (n_candidates) *n_candidates = c;
    return emit(all, out, cap);
}

/*
 * Algorithmic work of an execution plan, counted by replaying it (Section 5.1,
 * "Tree traversal on GPUs": the sequential path with a checkpoint per rule,
 * each distinct predicate evaluated once per pair and its result reused) on
 * every candidate pair, enumerated as in or_block_owned.  For a pair:
 *
 *   alive = the MDs whose equality predicates all hold; an alive MD without
 *   other predicates is a witness at once.  Then for each step k of prog
 *   (a predicate index into preds, one per distinct non-equality predicate,
 *   in plan order) whose MD set need[k] meets alive: evaluate it, and drop
 *   need[k] from alive when it fails; stop with a witness once an alive MD
 *   has its checkpoint at k (cp_step[m] == k, its last predicate), or with
 *   none once alive is empty.
 *
 * Units added (units_out, int64[7]): [0] n_eq_keys compares per candidate
 * pair; [1] n_md compares (owner check) per candidate pair; [2] 3 per
 * |a - b| <= delta; [3] edit distance: 3 for the length filter, and when
 * |la - lb| <= k also ceil(min(la, lb) / 64) * max(la, lb) * 16 (bit-parallel
 * distance over 64-bit words); [4] Jaccard: 3 for the size filter, and when
 * min(|A|,|B|) * den >= num * max(|A|,|B|) also (|A| + |B|) * 4 (merge
 * intersection); a missing operand costs the filter only.  [5] candidate
 * pairs; [6] pairs where the replayed verdict differs from the disjunction
 * (must be 0: the plan does not change the result).  Returns units_out[6].
 */
int64_t or_plan_units(int64_t nR, int32_t ncR, const or_col *R, int64_t nS, int32_t ncS, const or_col *S,
                      int32_t n_md, const int32_t *md_start, const or_pred *preds, int32_t n_threads,
                      int32_t n_eq_keys, int32_t n_prog, const int32_t *prog, const uint64_t *need,
                      const int32_t *cp_step, int64_t *units_out) {
    Rel r{nR, ncR, R};
    Rel s = S ? Rel{nS, ncS, S} : r;
    const bool self = (S == nullptr);
    const int nt = std::max(n_threads, 1);
    std::vector<std::vector<int64_t>> gid_r((size_t)n_md), gid_s((size_t)n_md);
    std::vector<std::vector<std::vector<int64_t>>> left((size_t)n_md), right((size_t)n_md);
    for (int m = 0; m < n_md; m++)
        group_ids(preds, md_start[m], md_start[m + 1], r, self ? nullptr : &s, gid_r[(size_t)m], gid_s[(size_t)m],
                  left[(size_t)m], right[(size_t)m]);
    const std::vector<std::vector<int64_t>> &gid_c = self ? gid_r : gid_s;
    std::vector<GramSets> grams;
    for (int k = 0; k < n_prog; k++) {
        const or_pred &p = preds[prog[k]];
        if (p.kind != 3) continue;
        for (int side = 0; side < (self ? 1 : 2); side++) {
            const int col = side == 0 ? p.col_t : p.col_s;
            bool have = false;
            for (const GramSets &g : grams) have = have || (g.side == side && g.col == col && g.q == p.q);
            if (have) continue;
            grams.push_back(GramSets{side, col, p.q, {}});
            gram_rows(side == 0 ? r : s, col, p.q, nt, grams.back().rows);
        }
    }
    Owned ev{n_md, md_start, preds, r, s, grams, self};
    struct Unit { int m; int64_t g, a0, a1; };
    std::vector<Unit> units;
    for (int m = 0; m < n_md; m++)
        for (size_t g = 0; g < left[(size_t)m].size(); g++) {
            const int64_t nl = (int64_t)left[(size_t)m][g].size();
            const int64_t nrt = self ? nl : (int64_t)right[(size_t)m][g].size();
            if (nl == 0 || nrt == 0 || (self && nl < 2)) continue;
            for (int64_t a = 0; a < nl;) {
                int64_t b = a, pairs = 0;
                while (b < nl && pairs < (1 << 20)) { pairs += self ? (nl - 1 - b) : nrt; b++; }
                units.push_back(Unit{m, (int64_t)g, a, b});
                a = b;
            }
        }
    std::vector<int64_t> eqonly((size_t)n_md);   /* MD has no non-equality predicate */
    for (int m = 0; m < n_md; m++) {
        eqonly[(size_t)m] = 1;
        for (int32_t k = md_start[m]; k < md_start[m + 1]; k++) if (!is_equality(preds[k])) eqonly[(size_t)m] = 0;
    }
    auto filter_and_work = [&](const or_pred &p, int64_t i, int64_t j) -> int64_t {
        const or_col &a = r.cols[p.col_t], &b = s.cols[p.col_s];
        if (!present(a, i) || !present(b, j)) return 3;
        if (p.kind == 2) {
            const int64_t la = (int64_t)(a.off[i + 1] - a.off[i]), lb = (int64_t)(b.off[j + 1] - b.off[j]);
            if (std::llabs(la - lb) > (int64_t)p.k) return 3;
            return 3 + ((std::min(la, lb) + 63) / 64) * std::max(la, lb) * 16;
        }
        const auto *A = ev.gram_of(0, p.col_t, p.q), *B = ev.gram_of(1, p.col_s, p.q);
        const int64_t na = (int64_t)(*A)[(size_t)i].size(), nb = (int64_t)(*B)[(size_t)j].size();
        if ((uint64_t)std::min(na, nb) * p.den < (uint64_t)p.num * (uint64_t)std::max(na, nb)) return 3;
        return 3 + (na + nb) * 4;
    };
    std::atomic<size_t> next{0};
    std::vector<std::array<int64_t, 7>> acc((size_t)nt);
    for (auto &x : acc) x.fill(0);
    auto work = [&](int t) {
        std::array<int64_t, 7> &u = acc[(size_t)t];
        for (;;) {
            const size_t w = next.fetch_add(1);
            if (w >= units.size()) break;
            const Unit &U = units[w];
            const std::vector<int64_t> &L = left[(size_t)U.m][(size_t)U.g];
            const std::vector<int64_t> &Rt = self ? L : right[(size_t)U.m][(size_t)U.g];
            for (int64_t a = U.a0; a < U.a1; a++)
                for (int64_t b = self ? a + 1 : 0; b < (int64_t)Rt.size(); b++) {
                    int64_t i = L[(size_t)a], j = Rt[(size_t)b];
                    if (self && i > j) std::swap(i, j);
                    bool owned = true;
                    for (int mm = 0; mm < U.m && owned; mm++) {
                        const int64_t x = gid_r[(size_t)mm][(size_t)i];
                        owned = !(x >= 0 && x == gid_c[(size_t)mm][(size_t)j]);
                    }
                    if (!owned) continue;
                    u[5]++;
                    u[0] += n_eq_keys;
                    u[1] += n_md;
                    uint64_t alive = 0;
                    bool hit = false;
                    for (int m = 0; m < n_md; m++) {
                        bool all = true;
                        for (int32_t k = md_start[m]; k < md_start[m + 1] && all; k++)
                            if (is_equality(preds[k])) all = holds(preds[k], r, i, s, j);
                        if (all) {
                            alive |= 1ull << m;
                            hit = hit || eqonly[(size_t)m];
                        }
                    }
                    for (int k = 0; k < n_prog && !hit && alive; k++) {
                        if (!(alive & need[k])) continue;
                        const or_pred &p = preds[prog[k]];
                        if (p.kind == 4) u[2] += 3;
                        else u[p.kind == 2 ? 3 : 4] += filter_and_work(p, i, j);
                        if (!ev.holds_p(p, i, j)) alive &= ~need[k];
                        for (int m = 0; m < n_md && !hit; m++)
                            hit = ((alive >> m) & 1ull) && cp_step[m] == k;
                    }
                    if (hit != ev.dnf(i, j)) u[6]++;
                }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; t++) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
    for (int f = 0; f < 7; f++) {
        units_out[f] = 0;
        for (int t = 0; t < nt; t++) units_out[f] += acc[(size_t)t][(size_t)f];
    }
    return units_out[6];
}

/* Disjunction verdict for given pairs (i << 32 | j); used for sampled checks at full size. */
void or_check_pairs(int64_t nR, int32_t ncR, const or_col *R, int64_t nS, int32_t ncS, const or_col *S,
                    int32_t n_md, const int32_t *md_start, const or_pred *preds, const uint64_t *pairs, int64_t n,
                    uint8_t *verdict) {
    Rel r{nR, ncR, R};
    Rel s = S ? Rel{nS, ncS, S} : r;
    for (int64_t k = 0; k < n; k++) {
        int64_t i = (int64_t)(pairs[k] >> 32), j = (int64_t)(pairs[k] & 0xffffffffu);
        verdict[k] = pair_holds(n_md, md_start, preds, r, i, s, j, S == nullptr, true) ? 1 : 0;
    }
}

/* Single-predicate verdicts (for the per-predicate logs and unit pins). */
void or_pred_verdicts(int64_t nR, int32_t ncR, const or_col *R, int64_t nS, int32_t ncS, const or_col *S,
                      const or_pred *pred, const uint64_t *pairs, int64_t n, uint8_t *verdict) {
    Rel r{nR, ncR, R};
    Rel s = S ? Rel{nS, ncS, S} : r;
    for (int64_t k = 0; k < n; k++) {
        int64_t i = (int64_t)(pairs[k] >> 32), j = (int64_t)(pairs[k] & 0xffffffffu);
        verdict[k] = holds(*pred, r, i, s, j) ? 1 : 0;
    }
}

}  // extern "C"
