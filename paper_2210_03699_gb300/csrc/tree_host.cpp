// Host side of the far-field acceleration (tree_host.hpp): octree, exact
// separation test, interaction lists, and the host-only C entry point
// ctr_farfield_plan.  No CUDA in this file.
#include "tree_host.hpp"

#include <algorithm>
#include <cmath>
#include <string>
#include <thread>

#include "ctr_ibim.h"

namespace ctr {

int fail(int status, const std::string& msg);

namespace tree {

void build_octree(const int32_t* ijk, int64_t M, int leaf, Octree& t) {
    t = Octree{};
    std::vector<int32_t> idx((size_t)M), tmp((size_t)M);
    for (int64_t i = 0; i < M; ++i) idx[(size_t)i] = (int32_t)i;
    std::vector<std::vector<int32_t>> kids;
    // cells are segments [a, b) of idx; a stable bucket split keeps every segment in increasing node order
    auto split = [&](auto&& self, int32_t a, int32_t b) -> int32_t {
        const int32_t cid = (int32_t)t.begin.size();
        int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        for (int32_t q = a; q < b; ++q)
            for (int c = 0; c < 3; ++c) {
                const int32_t v = ijk[3 * (int64_t)idx[q] + c];
                lo[c] = std::min(lo[c], v);
                hi[c] = std::max(hi[c], v + 1);
            }
        t.begin.push_back(a);
        t.end.push_back(b);
        for (int c = 0; c < 3; ++c) {
            t.lo.push_back(lo[c]);
            t.hi.push_back(hi[c]);
        }
        kids.emplace_back();
        if (b - a <= leaf) return cid;
        int32_t mid[3];
        bool cut[3];
        for (int c = 0; c < 3; ++c) {
            cut[c] = hi[c] - lo[c] >= 2;
            mid[c] = lo[c] + (hi[c] - lo[c]) / 2;
        }
        auto code = [&](int32_t node) {
            int v = 0;
            for (int c = 0; c < 3; ++c)
                if (cut[c] && ijk[3 * (int64_t)node + c] >= mid[c]) v |= 1 << c;
            return v;
        };
        int32_t cnt[9] = {0};
        for (int32_t q = a; q < b; ++q) cnt[code(idx[q]) + 1]++;
        for (int k = 0; k < 8; ++k) cnt[k + 1] += cnt[k];
        int32_t fill[8];
        for (int k = 0; k < 8; ++k) fill[k] = a + cnt[k];
        for (int32_t q = a; q < b; ++q) tmp[fill[code(idx[q])]++] = idx[q];
        std::copy(tmp.begin() + a, tmp.begin() + b, idx.begin() + a);
        std::vector<int32_t> ch;
        for (int k = 0; k < 8; ++k)
            if (cnt[k + 1] > cnt[k]) ch.push_back(self(self, a + cnt[k], a + cnt[k + 1]));
        kids[cid] = ch;
        return cid;
    };
    if (M > 0) split(split, 0, (int32_t)M);
    t.perm.swap(idx);
    t.child_ptr.assign(t.begin.size() + 1, 0);
    for (size_t c = 0; c < kids.size(); ++c) t.child_ptr[c + 1] = t.child_ptr[c] + (int32_t)kids[c].size();
    t.child.reserve(t.child_ptr.back());
    for (const auto& k : kids) t.child.insert(t.child.end(), k.begin(), k.end());
}

int theta_q(double theta) { return (int)std::floor(1024.0 * theta + 0.5); }

void widened(const int32_t lo[3], const int32_t hi[3], int g, int64_t c2[3], int64_t* R2) {
    int64_t r = 0;
    for (int a = 0; a < 3; ++a) {
        c2[a] = (int64_t)lo[a] + (int64_t)hi[a] - 1;
        const int64_t e = (int64_t)hi[a] - 1 - (int64_t)lo[a] + 2 * (int64_t)g;
        r += e * e;
    }
    *R2 = r;
}

bool separated(const int64_t cB[3], int64_t R2B, const int64_t cC[3], int64_t R2C, int tq) {
    int64_t D2 = 0;
    for (int a = 0; a < 3; ++a) {
        const int64_t d = cB[a] - cC[a];
        D2 += d * d;
    }
    const __int128 A = (__int128)tq * tq * D2 - ((__int128)1 << 20) * ((__int128)R2B + R2C);
    if (A <= 0) return false;
    return A * A > ((__int128)1 << 42) * (__int128)R2B * (__int128)R2C;
}

void interaction_lists(const Octree& t, const int32_t* ijk, const int32_t* excl_ptr, const int32_t* excl,
                       int BS, int tq, int64_t min_far, int g, Lists& L) {
    const int64_t M = (int64_t)t.perm.size();
    const int32_t nc = t.n_clusters();
    std::vector<int32_t> pos((size_t)M);
    for (int64_t p = 0; p < M; ++p) pos[(size_t)t.perm[(size_t)p]] = (int32_t)p;
    std::vector<int64_t> cc(3 * (size_t)nc), cr((size_t)nc);
    for (int32_t c = 0; c < nc; ++c) widened(&t.lo[3 * (size_t)c], &t.hi[3 * (size_t)c], g, &cc[3 * (size_t)c], &cr[c]);
    const int64_t nb = (M + BS - 1) / BS;
    std::vector<std::vector<int32_t>> near((size_t)nb), far((size_t)nb);
    auto one_block = [&](int64_t I) {
        const int64_t p0 = I * BS, p1 = std::min<int64_t>(M, p0 + BS);
        int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        std::vector<int32_t> ex;
        for (int64_t p = p0; p < p1; ++p) {
            const int32_t i = t.perm[(size_t)p];
            for (int c = 0; c < 3; ++c) {
                lo[c] = std::min(lo[c], ijk[3 * (int64_t)i + c]);
                hi[c] = std::max(hi[c], ijk[3 * (int64_t)i + c] + 1);
            }
            for (int32_t e = excl_ptr[i]; e < excl_ptr[i + 1]; ++e) ex.push_back(pos[(size_t)excl[e]]);
        }
        std::sort(ex.begin(), ex.end());
        ex.erase(std::unique(ex.begin(), ex.end()), ex.end());
        int64_t cB[3], R2B;
        widened(lo, hi, g, cB, &R2B);
        auto holds_excluded = [&](int32_t c) {
            auto it = std::lower_bound(ex.begin(), ex.end(), t.begin[c]);
            return it != ex.end() && *it < t.end[c];
        };
        std::vector<int32_t>& nr = near[(size_t)I];
        std::vector<int32_t>& fr = far[(size_t)I];
        auto add_near = [&](int32_t b, int32_t e) {
            if (!nr.empty() && nr.back() == b) nr.back() = e;
            else {
                nr.push_back(b);
                nr.push_back(e);
            }
        };
        std::vector<int32_t> stack{0};
        while (!stack.empty()) {
            const int32_t c = stack.back();
            stack.pop_back();
            const bool leafc = t.child_ptr[c + 1] == t.child_ptr[c];
            if (separated(cB, R2B, &cc[3 * (size_t)c], cr[c], tq) && !holds_excluded(c)) {
                if ((int64_t)(t.end[c] - t.begin[c]) > min_far) fr.push_back(c);
                else add_near(t.begin[c], t.end[c]);
            } else if (leafc) {
                add_near(t.begin[c], t.end[c]);
            } else {
                for (int32_t k = t.child_ptr[c + 1] - 1; k >= t.child_ptr[c]; --k) stack.push_back(t.child[k]);
            }
        }
    };
    if (M > 0) {
        const int nthreads = (int)std::max<int64_t>(
            1, std::min<int64_t>({(int64_t)std::max(1u, std::thread::hardware_concurrency()), 16, nb}));
        std::vector<std::thread> pool;
        for (int w = 0; w < nthreads; ++w)
            pool.emplace_back([&, w]() {
                for (int64_t I = w; I < nb; I += nthreads) one_block(I);
            });
        for (auto& th : pool) th.join();
    }
    L = Lists{};
    L.BS = BS;
    L.near_ptr.assign((size_t)nb + 1, 0);
    L.far_ptr.assign((size_t)nb + 1, 0);
    for (int64_t I = 0; I < nb; ++I) {
        L.near_ptr[I + 1] = L.near_ptr[I] + (int64_t)near[(size_t)I].size() / 2;
        L.far_ptr[I + 1] = L.far_ptr[I] + (int64_t)far[(size_t)I].size();
        L.near_rng.insert(L.near_rng.end(), near[(size_t)I].begin(), near[(size_t)I].end());
        L.far_cl.insert(L.far_cl.end(), far[(size_t)I].begin(), far[(size_t)I].end());
    }
}

}  // namespace tree
}  // namespace ctr

extern "C" int ctr_farfield_plan(int64_t M, const int32_t* ijk, const int32_t* excl_ptr, const int32_t* excl,
                                 int margin, int degree, double theta, int leaf, int block, int64_t min_far,
                                 int64_t* perm,
                                 int64_t* n_near_ranges, int64_t* n_far, int64_t* near_ptr, int64_t* near_rng,
                                 int64_t* far_ptr, int64_t* far_begin, int64_t* far_end) {
    using namespace ctr;
    try {
        if (M <= 0 || !ijk || !excl_ptr || !excl) return fail(CTR_ERR_INVALID, "farfield plan: bad nodes");
        if (M > INT32_MAX / 4) return fail(CTR_ERR_CAPACITY, "farfield plan: too many nodes");
        if (degree < 2 || degree > 12 || leaf < 1 || block < 1 || margin < 0 || !(theta >= 0.0 && theta < 1.0))
            return fail(CTR_ERR_INVALID, "farfield plan: bad parameters");
        if (margin > (1 << 20)) return fail(CTR_ERR_INVALID, "farfield plan: margin must be <= 2^20");
        // the caller's arrays are read as given: check them before any of them indexes another
        for (int64_t k = 0; k < 3 * M; ++k)
            if (ijk[k] <= -(1 << 30) || ijk[k] >= (1 << 30))
                return fail(CTR_ERR_INVALID, "farfield plan: grid indices must lie in (-2^30, 2^30)");
        if (excl_ptr[0] != 0) return fail(CTR_ERR_INVALID, "farfield plan: excl_ptr[0] must be 0");
        for (int64_t i = 0; i < M; ++i)
            if (excl_ptr[i + 1] < excl_ptr[i]) return fail(CTR_ERR_INVALID, "farfield plan: excl_ptr must not decrease");
        for (int64_t e = 0; e < (int64_t)excl_ptr[M]; ++e)
            if (excl[e] < 0 || (int64_t)excl[e] >= M)
                return fail(CTR_ERR_INVALID, "farfield plan: excluded node out of range");
        tree::Octree t;
        tree::build_octree(ijk, M, leaf, t);
        tree::Lists L;
        const int64_t np = (int64_t)(degree + 1) * (degree + 1) * (degree + 1);
        tree::interaction_lists(t, ijk, excl_ptr, excl, block, tree::theta_q(theta), min_far > 0 ? min_far : np,
                                margin, L);
        const int64_t nb = (int64_t)L.near_ptr.size() - 1;
        if (perm)
            for (int64_t p = 0; p < M; ++p) perm[p] = t.perm[(size_t)p];
        if (n_near_ranges) *n_near_ranges = L.near_ptr.back();
        if (n_far) *n_far = L.far_ptr.back();
        if (near_ptr)
            for (int64_t I = 0; I <= nb; ++I) near_ptr[I] = L.near_ptr[(size_t)I];
        if (far_ptr)
            for (int64_t I = 0; I <= nb; ++I) far_ptr[I] = L.far_ptr[(size_t)I];
        if (near_rng)
            for (size_t k = 0; k < L.near_rng.size(); ++k) near_rng[k] = L.near_rng[k];
        for (size_t k = 0; k < L.far_cl.size(); ++k) {
            if (far_begin) far_begin[k] = t.begin[(size_t)L.far_cl[k]];
            if (far_end) far_end[k] = t.end[(size_t)L.far_cl[k]];
        }
        return CTR_OK;
    } catch (...) {
        return fail(CTR_ERR_NOMEM, "farfield plan: host allocation failed");
    }
}
