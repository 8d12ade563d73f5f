// Far-field acceleration of the dense sum (Sec. 2.5): the treecode of one
// handle.  Setup (once): the octree and interaction lists (tree_host.cpp),
// the nodes' tree order (the packed source arrays are permuted to it, so that
// every cluster and target block is a contiguous range), the exclusion lists
// in tree positions, and per pair arithmetic the schedule: one-sided pair
// items for the direct ("near") ranges, far items for the far clusters and the
// moment chunks of the clusters that carry charges; near and far items add
// their sums into the nodes' exact accumulators (order-independent).  Per
// operator application: the near items run in the
// pair kernels like any schedule; launch_tree runs the moments, the charge
// reduction and the far items (tree.cuh).
#include <cmath>
#include <mutex>
#include <numeric>

#include "tree.cuh"
#include "tree_host.hpp"

namespace ctr {

using namespace pk;

namespace {

constexpr int kTreeItemsPerSlot = 4;
// A well-separated cluster is approximated when it has more than (degree+1)^3 / kMinFarDiv nodes: a
// float-float pair costs about two float-float proxy evaluations, an FP32 or FP64 pair about one.
constexpr int kMinFarDiv[3] = {1, 2, 1};
// Cost of one proxy evaluation relative to one one-sided pair of the arithmetic (item splitting only).
constexpr double kFarCost[3] = {0.4, 0.45, 0.5};

template <typename T>
__global__ void gather_rows(const T* __restrict__ src, T* __restrict__ dst, const int32_t* __restrict__ perm,
                            int64_t M, int per) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M * per) return;
    const int64_t p = k / per, c = k % per;
    dst[k] = src[(int64_t)perm[p] * per + c];
}

template <typename T>
int permute_rows(DevBuf& buf, const DevBuf& d_perm, int64_t M, int per, cudaStream_t st) {
    DevBuf tmp;
    CTR_TRY(tmp.alloc(sizeof(T) * (size_t)M * per));
    CTR_CUDA_TRY(cudaMemcpyAsync(tmp.p, buf.p, sizeof(T) * (size_t)M * per, cudaMemcpyDeviceToDevice, st));
    gather_rows<T><<<grid_for(M * per, 256), 256, 0, st>>>(tmp.as<T>(), buf.as<T>(), d_perm.as<int32_t>(), M, per);
    CTR_LAUNCHED();
    CTR_CUDA_TRY(cudaStreamSynchronize(st));   // tmp is released on return
    return CTR_OK;
}

template <typename T>
int upload(DevBuf& d, const std::vector<T>& h, cudaStream_t st) {
    CTR_TRY(d.alloc(sizeof(T) * std::max<size_t>(1, h.size())));
    if (!h.empty()) CTR_CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
    return CTR_OK;
}

template <typename T>
int download(std::vector<T>& h, const void* d, size_t n, cudaStream_t st) {
    h.resize(n);
    if (n) CTR_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
    return CTR_OK;
}



template <typename Real, int R, int NT>
int launch_tree_t(ctr_ibim* s, int pol) {
    TreeData& t = *s->tree;
    TreeData::Pol& P = t.pol[pol];
    if (P.far.empty()) return CTR_OK;
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    cudaStream_t st = s->stream;
    const OneTreeAcc acc{t.d_view.as<TreeView>()};
    int* counters = t.d_counters.as<int>() + 2 * pol;
    const int* counts = t.d_counters.as<int>() + 6 + 3 * pol;
    CTR_CUDA_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(int), st));
    const int nchunks = (int)P.chunks.size();
    k_tree_mom<Real, OneTreeAcc><<<std::min(2 * sms, nchunks), kThreads, 0, st>>>(
        acc, P.d_ent_mom.as<int2>(), counts, counters, pol);
    CTR_LAUNCHED();
    k_tree_momred<Real, OneTreeAcc><<<std::min(4 * sms, P.nq), kThreads, 0, st>>>(acc, P.d_ent_red.as<int2>(),
                                                                                counts + 1, pol);
    CTR_LAUNCHED();
    if (R * NT != s->sched[pol].BS) return fail(CTR_ERR_INVALID, "treecode: far kernel shape != target block");
    static std::map<std::pair<int, int>, int> cache;
    if constexpr (sizeof(Real) == 8 && R == kTreeR[1] && NT == kTreeNT[1]) {   // float-float far field
        auto kern = k_tree_far_ff<R, NT, OneTreeAcc>;
        const int smem = (int)tree_farff_smem(P.np);
        const int per_sm = far_per_sm(kern, NT, smem, (int)tree_farff_smem(), cache);
        if (per_sm < 0) return per_sm;
        kern<<<std::min<int64_t>((int64_t)per_sm * sms, (int64_t)P.far.size()), NT, smem, st>>>(
            acc, P.d_ent_far.as<int2>(), counts + 2, counters + 1);
    } else if constexpr (sizeof(Real) == 4) {
        auto kern = k_tree_far2<R / 2, NT, OneTreeAcc>;
        const int smem = (int)tree_far2_smem(P.np);
        const int per_sm = far_per_sm(kern, NT, smem, (int)tree_far2_smem(), cache);
        if (per_sm < 0) return per_sm;
        kern<<<std::min<int64_t>((int64_t)per_sm * sms, (int64_t)P.far.size()), NT, smem, st>>>(
            acc, P.d_ent_far.as<int2>(), counts + 2, counters + 1, pol);
    } else {
        auto kern = k_tree_far<Real, R, NT, OneTreeAcc>;
        const int per_sm = far_per_sm(kern, NT, (int)tree_far_smem<Real>(), (int)tree_far_smem<Real>(), cache);
        if (per_sm < 0) return per_sm;
        kern<<<std::min<int64_t>((int64_t)per_sm * sms, (int64_t)P.far.size()), NT, tree_far_smem<Real>(), st>>>(
            acc, P.d_ent_far.as<int2>(), counts + 2, counters + 1, pol);
    }
    CTR_LAUNCHED();
    return CTR_OK;
}

}  // namespace

int launch_tree(ctr_ibim* s, int pol) {
    if (!s->tree) return CTR_OK;
    if (pol == 0) return launch_tree_t<float, kTreeR[0], kTreeNT[0]>(s, 0);
    if (pol == 1) return launch_tree_t<double, kTreeR[1], kTreeNT[1]>(s, 1);
    return launch_tree_t<double, kTreeR[2], kTreeNT[2]>(s, 2);
}

int64_t tree_bytes(const ctr_ibim* s) {
    if (!s->tree) return 0;
    const TreeData& t = *s->tree;
    int64_t b = (int64_t)(t.d_tinv.bytes + t.d_eptr.bytes + t.d_excl.bytes + t.d_counters.bytes + t.d_view.bytes);
    for (const auto& P : t.pol)
        b += (int64_t)(P.d_xref.bytes + P.d_bw.bytes + P.d_dref.bytes + P.d_box.bytes + P.d_chunks.bytes +
                       P.d_cptr.bytes + P.d_mpart.bytes + P.d_mom.bytes + P.d_far.bytes + P.d_flist.bytes +
                       P.d_ent_mom.bytes + P.d_ent_red.bytes + P.d_ent_far.bytes);
    return b;
}

int build_tree_schedules(ctr_ibim* s, const int slots[3]) {
    const int64_t M = s->M;
    cudaStream_t st = s->stream;
    if (M > INT32_MAX / 4) return fail(CTR_ERR_CAPACITY, "treecode: too many nodes");
    auto T = std::make_unique<TreeData>();
    TreeData& t = *T;
    t.leaf = s->opt.tree_leaf;
    t.g = (int)std::ceil(s->eps / s->h);
    for (int p = 0; p < 3; ++p) {   // the FP32 operator (inner GMRES) has its own degree and theta
        TreeData::Pol& P = t.pol[p];
        P.degree = p == 0 ? s->opt.tree_degree_fp32 : s->opt.tree_degree;
        P.theta = p == 0 ? s->opt.tree_theta_fp32 : s->opt.tree_theta;
        P.n1 = P.degree + 1;
        P.np = P.n1 * P.n1 * P.n1;
    }
    // ---- node indices, closest points, correction sets (host copies)
    std::vector<int64_t> lin;
    std::vector<double> Px, Py, Pz;
    std::vector<int32_t> cptr, excl;
    CTR_TRY(download(lin, s->lin.p, (size_t)M, st));
    CTR_TRY(download(Px, s->na.Px, (size_t)M, st));
    CTR_TRY(download(Py, s->na.Py, (size_t)M, st));
    CTR_TRY(download(Pz, s->na.Pz, (size_t)M, st));
    CTR_TRY(download(cptr, s->corr_ptr.p, (size_t)M + 1, st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    CTR_TRY(download(excl, s->excl.p, (size_t)cptr[(size_t)M], st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> ijk(3 * (size_t)M);
    for (int64_t i = 0; i < M; ++i) {
        const int64_t l = lin[(size_t)i];
        ijk[3 * (size_t)i] = (int32_t)(l % s->n[0]);
        ijk[3 * (size_t)i + 1] = (int32_t)((l / s->n[0]) % s->n[1]);
        ijk[3 * (size_t)i + 2] = (int32_t)(l / (s->n[0] * s->n[1]));
    }
    tree::Octree oct;
    tree::build_octree(ijk.data(), M, t.leaf, oct);
    t.perm = oct.perm;
    t.n_clusters = oct.n_clusters();
    std::vector<int32_t> pos((size_t)M);
    for (int64_t p = 0; p < M; ++p) pos[(size_t)oct.perm[(size_t)p]] = (int32_t)p;
    // ---- exclusion CSR in tree positions
    std::vector<int32_t> teptr((size_t)M + 1, 0), texcl(excl.size());
    for (int64_t p = 0; p < M; ++p) {
        const int32_t i = oct.perm[(size_t)p];
        const int32_t n = cptr[(size_t)i + 1] - cptr[(size_t)i];
        teptr[(size_t)p + 1] = teptr[(size_t)p] + n;
        for (int32_t e = 0; e < n; ++e) texcl[(size_t)teptr[(size_t)p] + e] = pos[(size_t)excl[(size_t)cptr[(size_t)i] + e]];
        std::sort(texcl.begin() + teptr[(size_t)p], texcl.begin() + teptr[(size_t)p + 1]);
    }
    CTR_TRY(upload(t.d_tinv, pos, st));
    CTR_TRY(upload(t.d_eptr, teptr, st));
    CTR_TRY(upload(t.d_excl, texcl, st));
    // ---- sources in tree order
    DevBuf d_perm;
    CTR_TRY(upload(d_perm, oct.perm, st));
    CTR_TRY(permute_rows<float4>(s->src32, d_perm, M, 4, st));
    CTR_TRY(permute_rows<double4>(s->src64, d_perm, M, 2, st));
    CTR_TRY(permute_rows<float4>(s->srcdf, d_perm, M, 4, st));
    // ---- per arithmetic: Chebyshev points of the second kind, barycentric weights, differentiation matrix
    for (int p = 0; p < 3; ++p) {
        TreeData::Pol& P = t.pol[p];
        const int n = P.degree, n1 = P.n1;
        std::vector<double> xr(n1), bw(n1), dr((size_t)n1 * n1, 0.0);
        for (int m = 0; m < n1; ++m) {
            xr[m] = std::cos(kPi * m / n);
            bw[m] = ((m % 2) ? -1.0 : 1.0) * ((m == 0 || m == n) ? 0.5 : 1.0);
        }
        for (int m = 0; m < n1; ++m) {
            double diag = 0.0;
            for (int q = 0; q < n1; ++q)
                if (q != m) {
                    dr[(size_t)m * n1 + q] = (bw[q] / bw[m]) / (xr[m] - xr[q]);
                    diag += dr[(size_t)m * n1 + q];
                }
            dr[(size_t)m * n1 + m] = -diag;
        }
        CTR_TRY(upload(P.d_xref, xr, st));
        CTR_TRY(upload(P.d_bw, bw, st));
        CTR_TRY(upload(P.d_dref, dr, st));
        CTR_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // ---- per pair arithmetic: lists, items, chunks
    const int Rs[3] = {kR32 * Fp32x2Policy::kPack, kRdf, kR64};
    const int tiles[3] = {Fp32x2Policy::kTile, Df64Policy::kTile, Fp64Policy::kTile};
    const size_t real_bytes[3] = {sizeof(float), sizeof(double), sizeof(double)};   // moments and charges
    std::vector<int> counts(15, 0);
    for (int p = 0; p < 3; ++p) {
        PairSchedule& sc = s->sched[p];
        TreeData::Pol& P = t.pol[p];
        sc.items.clear();
        sc.cost.clear();
        sc.R = Rs[p];
        sc.BS = kThreads * Rs[p];
        sc.tile = tiles[p];
        const int BS = sc.BS;
        if (BS != kTreeR[p] * kTreeNT[p]) return fail(CTR_ERR_INVALID, "treecode: far kernel shape != target block");
        const int nb = (int)((M + BS - 1) / BS);
        sc.nb = nb;
        tree::Lists L;
        tree::interaction_lists(oct, ijk.data(), cptr.data(), excl.data(), BS, tree::theta_q(P.theta),
                                (int64_t)(P.np / kMinFarDiv[p]), t.g, L);
        // far clusters that carry charges, in increasing cluster id
        std::vector<int32_t> ids(L.far_cl);
        std::sort(ids.begin(), ids.end());
        ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
        std::vector<int32_t> compact((size_t)oct.n_clusters(), -1);
        for (size_t q = 0; q < ids.size(); ++q) compact[(size_t)ids[q]] = (int32_t)q;
        P.nq = (int)ids.size();
        std::vector<double> box(6 * ids.size());
        std::vector<int32_t> ccp(ids.size() + 1, 0);
        P.chunks.clear();
        P.chunk_cost.clear();
        for (size_t q = 0; q < ids.size(); ++q) {
            const int32_t c = ids[q];
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int32_t pp = oct.begin[(size_t)c]; pp < oct.end[(size_t)c]; ++pp) {
                const int32_t i = oct.perm[(size_t)pp];
                const double v[3] = {Px[(size_t)i], Py[(size_t)i], Pz[(size_t)i]};
                for (int a = 0; a < 3; ++a) {
                    lo[a] = std::min(lo[a], v[a]);
                    hi[a] = std::max(hi[a], v[a]);
                }
            }
            for (int a = 0; a < 3; ++a) {
                box[6 * q + a] = 0.5 * (lo[a] + hi[a]);
                box[6 * q + 3 + a] = std::max(0.5 * (hi[a] - lo[a]), s->h / 1024.0);
            }
            for (int32_t j0 = oct.begin[(size_t)c]; j0 < oct.end[(size_t)c]; j0 += kChunkSrc) {
                const int32_t j1 = std::min<int32_t>(oct.end[(size_t)c], j0 + kChunkSrc);
                P.chunks.push_back(MomChunk{(int32_t)q, j0, j1, 0});
                P.chunk_cost.push_back((double)(j1 - j0));
            }
            ccp[q + 1] = (int32_t)P.chunks.size();
        }
        // near items (one-sided pair items over tree positions) and far items, with their regions
        double near_total = 0.0, far_total = 0.0;
        for (int I = 0; I < nb; ++I) {
            for (int64_t r = L.near_ptr[(size_t)I]; r < L.near_ptr[(size_t)I + 1]; ++r)
                near_total += (double)BS * (L.near_rng[2 * (size_t)r + 1] - L.near_rng[2 * (size_t)r]);
            far_total += (double)BS * P.np * kFarCost[p] * (double)(L.far_ptr[(size_t)I + 1] - L.far_ptr[(size_t)I]);
        }
        const double near_cmax = std::max(1.0, near_total / ((double)kTreeItemsPerSlot * std::max(1, slots[p])));
        const double far_cmax = std::max(1.0, far_total / ((double)kTreeItemsPerSlot * std::max(1, slots[p])));
        std::vector<PairItem> items;
        std::vector<double> icost;
        std::vector<int32_t> flist;
        P.far.clear();
        P.far_cost.clear();
        P.near_pairs = P.far_evals = P.far_pairs = 0;
        for (int I = 0; I < nb; ++I) {
            const int64_t nt = std::min<int64_t>(BS, M - (int64_t)I * BS);
            for (int64_t r = L.near_ptr[(size_t)I]; r < L.near_ptr[(size_t)I + 1]; ++r) {
                const int32_t b = L.near_rng[2 * (size_t)r], e = L.near_rng[2 * (size_t)r + 1];
                const int64_t len = e - b;
                P.near_pairs += nt * len;
                int64_t pieces = std::max<int64_t>(1, (int64_t)std::ceil((double)BS * len / near_cmax));
                int64_t plen = (len + pieces - 1) / pieces;
                plen = ((plen + tiles[p] - 1) / tiles[p]) * tiles[p];
                plen = std::max<int64_t>(plen, std::min<int64_t>(len, 2 * (int64_t)tiles[p]));
                for (int64_t a = b; a < e; a += plen) {
                    PairItem it{};
                    it.I = I;
                    it.j_begin = (int32_t)a;
                    it.j_end = (int32_t)std::min<int64_t>(e, a + plen);
                    it.sym = 0;
                    items.push_back(it);
                    icost.push_back((double)BS * (it.j_end - it.j_begin));
                }
            }
        }
        for (int I = 0; I < nb; ++I) {
            const int64_t nt = std::min<int64_t>(BS, M - (int64_t)I * BS);
            const int64_t f0 = L.far_ptr[(size_t)I], f1 = L.far_ptr[(size_t)I + 1];
            P.far_pairs += f1 - f0;
            P.far_evals += nt * (f1 - f0) * P.np;
            const double unit = (double)BS * P.np * kFarCost[p];
            const int64_t per_item = std::max<int64_t>(1, (int64_t)std::floor(far_cmax / unit));
            for (int64_t a = f0; a < f1; a += per_item) {
                const int64_t b = std::min<int64_t>(f1, a + per_item);
                FarItem fi{};
                fi.I = I;
                fi.l0 = (int32_t)flist.size();
                for (int64_t k = a; k < b; ++k) flist.push_back(compact[(size_t)L.far_cl[(size_t)k]]);
                fi.l1 = (int32_t)flist.size();
                P.far.push_back(fi);
                P.far_cost.push_back(unit * (double)(b - a));
            }
        }
        sc.pairs_one = P.near_pairs;
        sc.pairs_sym = 0;
        sc.total_cost = near_total;
        sc.planned = true;
        // near items in decreasing cost (the host copy follows the device order)
        std::vector<int> order(items.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return icost[a] > icost[b]; });
        sc.items.resize(items.size());
        sc.cost.resize(items.size());
        for (size_t k = 0; k < order.size(); ++k) {
            sc.items[k] = items[(size_t)order[k]];
            sc.cost[k] = icost[(size_t)order[k]];
        }
        CTR_TRY(upload(sc.d_items, sc.items, st));
        // far-field buffers and the single-system work entries (decreasing cost)
        CTR_TRY(upload(P.d_box, box, st));
        CTR_TRY(upload(P.d_chunks, P.chunks, st));
        CTR_TRY(upload(P.d_cptr, ccp, st));
        CTR_TRY(upload(P.d_far, P.far, st));
        CTR_TRY(upload(P.d_flist, flist, st));
        CTR_TRY(P.d_mpart.alloc(real_bytes[p] * 2 * (size_t)P.np * std::max<size_t>(1, P.chunks.size())));
        CTR_TRY(P.d_mom.alloc(real_bytes[p] * 3 * (size_t)P.np * std::max<size_t>(1, ids.size())));
        auto entries = [](const std::vector<double>& cost) {
            std::vector<int> o(cost.size());
            std::iota(o.begin(), o.end(), 0);
            std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return cost[a] > cost[b]; });
            std::vector<int2> e(o.size());
            for (size_t k = 0; k < o.size(); ++k) e[k] = make_int2(0, o[k]);
            return e;
        };
        std::vector<int2> red(ids.size());
        for (size_t q = 0; q < ids.size(); ++q) red[q] = make_int2(0, (int)q);
        CTR_TRY(upload(P.d_ent_mom, entries(P.chunk_cost), st));
        CTR_TRY(upload(P.d_ent_red, red, st));
        CTR_TRY(upload(P.d_ent_far, entries(P.far_cost), st));
        counts[3 * p] = (int)P.chunks.size();
        counts[3 * p + 1] = P.nq;
        counts[3 * p + 2] = (int)P.far.size();
        CTR_CUDA_TRY(cudaStreamSynchronize(st));   // host vectors of this pass go out of scope
    }
    CTR_TRY(alloc_accumulators(s));
    CTR_TRY(s->counter.alloc(sizeof(int) * 4));
    // counters: [2 per arithmetic] work counters, then [3 per arithmetic] entry counts
    std::vector<int> cnt(15, 0);
    for (int p = 0; p < 3; ++p)
        for (int k = 0; k < 3; ++k) cnt[6 + 3 * p + k] = counts[3 * p + k];
    CTR_TRY(upload(t.d_counters, cnt, st));
    // the device view
    TreeView& v = t.view;
    v.on = 1;
    v.M = (int)M;
    v.tinv = t.d_tinv.as<int32_t>();
    for (int p = 0; p < 3; ++p) {
        TreeData::Pol& P = t.pol[p];
        v.n1[p] = P.n1;
        v.np[p] = P.np;
        v.xref[p] = P.d_xref.as<double>();
        v.bw[p] = P.d_bw.as<double>();
        v.dref[p] = P.d_dref.as<double>();
        v.box[p] = P.d_box.as<double>();
        v.chunks[p] = P.d_chunks.as<MomChunk>();
        v.cptr[p] = P.d_cptr.as<int32_t>();
        v.mpart[p] = P.d_mpart.p;
        v.mom[p] = P.d_mom.p;
        v.far[p] = P.d_far.as<FarItem>();
        v.flist[p] = P.d_flist.as<int32_t>();
        v.BS[p] = s->sched[p].BS;
    }
    CTR_TRY(exp_table(s->device, &v.exp_tab));
    v.src32 = s->src32.as<float4>();
    v.srcdf = s->srcdf.as<float4>();
    v.src64 = s->src64.as<double4>();
    v.acc = s->acc.as<unsigned long long>();
    v.c1 = s->eps_out / s->eps_in;
    v.c2 = s->eps_in / s->eps_out;
    v.kappa = s->kappa;
    CTR_TRY(t.d_view.alloc(sizeof(TreeView)));
    CTR_CUDA_TRY(cudaMemcpyAsync(t.d_view.p, &v, sizeof(TreeView), cudaMemcpyHostToDevice, st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    s->tree = std::move(T);
    return CTR_OK;
}

}  // namespace ctr
