// Batched exact Hankel products: many matrices of different order and
// precision, each with a block of right-hand sides (as in block Lanczos),
// advanced together by one CUDA graph launch per call.
//
// Every (matrix, right-hand side) pair is one leaf problem of Algorithm 1
// (Beliakov, arXiv:1402.5287, Sec. 3).  The leaf products of all pairs of a
// wave run in ONE persistent tensor-core launch over a combined tile list
// (each tile names its problem; each problem carries its own TMA
// descriptors); the level kernels of all pairs run around it.  Pairs are
// grouped into waves so that the per-pair leaf operands and outputs of one
// wave fit a memory budget; level and post-pass buffers are shared by all
// pairs, since they are used one pair after another.  The whole sequence
// (every wave, every pair, the rounding of every matrix) is captured once in
// a CUDA graph and replayed by each hmv_batch_matvec.
//
// Members whose mantissas the cost model splits (Karatsuba or Toom-Cook on
// the digits, the same choice a single HMV_AUTO plan makes) keep their own
// buffers, outside the wave budget: they run in rounds, one per right-hand
// side, each round the vector side of every such member, ONE persistent leaf
// launch over all their digit products (per tile width), and the post-pass
// with the interpolation of every member.  Members on the exact NTT path
// (method HMV_NTT) keep their own buffers too and run their transforms, one
// right-hand side after another, in the same graph.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include "hmv_internal.h"

namespace hmv {
namespace {

struct Pair {
    int plan, rhs, wave;
    uint16_t *xg;
    uint8_t *dig;
    int32_t *carry;
};

}  // namespace
}  // namespace hmv

struct hmv_batch_s {
    cudaStream_t stream = nullptr;
    std::vector<hmv_plan_s *> plans;
    std::vector<hmv::Pair> pairs;
    int nwaves = 0;
    std::vector<hmv::LeafProblem *> d_probs;  // per wave
    std::vector<hmv::Tile *> d_tiles;         // per wave
    std::vector<int> ntiles;                  // per wave
    std::vector<int> wave_tn;                 // tile width of each wave's leaf launch
    std::vector<void *> allocations;
    int8_t *a_lvl[2] = {nullptr, nullptr}, *x_lvl[2] = {nullptr, nullptr};
    int32_t *post[2] = {nullptr, nullptr};
    int64_t device_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    bool own_stream = false;
    double leaf_macs = 0;
    int64_t tiles_total = 0;
    int64_t graph_launches = 0, kernels_per_launch = 0;
    int num_sms = 0;
    // members run as split plans (own buffers), and per round r (right-hand
    // side r) and tile width the combined leaf problems of their products
    std::vector<char> split;
    int split_rounds = 0;
    struct SplitLaunch {
        int round, tn, ntiles;
        hmv::LeafProblem *probs;
        hmv::Tile *tiles;
    };
    std::vector<SplitLaunch> split_launches;
    hmv_plan_s *split_first = nullptr;  // status word and tile counter of the split launches
    hmv_plan_s *wave_first = nullptr;   // the same for the waves' launches (a member run in waves)
    std::vector<char> ntt;              // members on the exact NTT path (own buffers, no leaf products)
    // parallel branches of the captured graph for the NTT members: side
    // streams that fork from and join back to `stream` during the capture
    std::vector<cudaStream_t> side;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
};

namespace hmv {
namespace {

cudaError_t balloc(hmv_batch_s *B, void **ptr, size_t bytes) {
    *ptr = nullptr;
    cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 1);
    if (e == cudaSuccess) {
        B->allocations.push_back(*ptr);
        B->device_bytes += static_cast<int64_t>(bytes);
    }
    return e;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Parallel branches of a batch graph for its NTT members.
constexpr int kNttBranches = 8;

size_t pair_bytes(const hmv_plan_s *p) {
    return align256(p->elems_xg * 2) + align256(p->bytes_dig) + align256(p->elems_carry * 4);
}

// Point a plan's working buffers at a pair's and the batch's shared ones.
void bind(hmv_batch_s *B, hmv_plan_s *p, const Pair &pr) {
    p->x_lvl[0] = B->x_lvl[0];
    p->x_lvl[1] = B->x_lvl[1];
    p->post[0] = B->post[0];
    p->post[1] = B->post[1];
    p->xg = pr.xg;
    p->leaf_dig = pr.dig;
    p->leaf_carry = pr.carry;
}

// The whole batched product, issued on B->stream (captured into a graph).
cudaError_t issue(hmv_batch_s *B) {
    cudaError_t e = cudaSuccess;
    int64_t kernels = 0;
    for (hmv_plan_s *p : B->plans) {
        if (e == cudaSuccess) e = cudaMemsetAsync(p->dstat, 0, 8 * sizeof(int32_t), B->stream);
        if (e == cudaSuccess) e = launch_validate(p, p->x_limbs_d, p->n * p->nrhs);
        ++kernels;
    }
    for (int w = 0; w < B->nwaves && e == cudaSuccess; ++w) {
        for (const Pair &pr : B->pairs) {
            if (pr.wave != w || e != cudaSuccess) continue;
            hmv_plan_s *p = B->plans[pr.plan];
            bind(B, p, pr);
            const uint32_t *xr = p->x_limbs_d + static_cast<size_t>(pr.rhs) * p->n * p->L32;
            const uint8_t *xnr = p->x_neg_d + static_cast<size_t>(pr.rhs) * p->n;
            e = launch_encode(p, xr, xnr, p->n, 0, p->x_lvl[0]);
            for (int l = 0; l < p->L && e == cudaSuccess; ++l)
                e = launch_prepass(p, l, false, p->x_lvl[l % 2], p->x_lvl[(l + 1) % 2]);
            if (e == cudaSuccess) e = launch_pack_vector(p, p->x_lvl[p->L % 2]);
            kernels += 2 + p->L;
        }
        if (e == cudaSuccess)
            e = launch_leaf_tc_multi(B->d_probs[w], B->d_tiles[w], B->ntiles[w], B->wave_first->dstat,
                                     B->wave_first->d_counter, B->stream, B->num_sms, B->wave_tn[w]);
        ++kernels;
        for (const Pair &pr : B->pairs) {
            if (pr.wave != w || e != cudaSuccess) continue;
            hmv_plan_s *p = B->plans[pr.plan];
            bind(B, p, pr);
            e = launch_post_group(&p, 1);  // leaf normalise and every post-pass level
            if (e == cudaSuccess) e = launch_final_normalize(p, p->post[0], pr.rhs, p->post16 ? 2 : 4);
            kernels += 1 + std::max(p->L, 1);
        }
    }
    // NTT members: transforms, pointwise product and extraction per right-hand
    // side, then the rounding, each member on one of the side streams (longest
    // first onto the least loaded branch, by transform work): the graph gets
    // parallel branches, so the short kernels of different members overlap
    // on the device instead of running one after another
    std::vector<int> nttm;
    for (size_t i = 0; i < B->plans.size(); ++i)
        if (B->ntt[i]) nttm.push_back(static_cast<int>(i));
    if (!nttm.empty() && e == cudaSuccess) {
        auto work = [&](int i) {
            const hmv_plan_s *p = B->plans[i];
            return static_cast<double>(p->nrhs) * static_cast<double>(p->ntt_N) * p->ntt_K;
        };
        std::stable_sort(nttm.begin(), nttm.end(), [&](int a, int b) { return work(a) > work(b); });
        const int nb = static_cast<int>(std::min(B->side.size(), nttm.size()));
        e = cudaEventRecord(B->fork_ev, B->stream);
        for (int j = 0; j < nb && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(B->side[j], B->fork_ev, 0);
        std::vector<double> load(nb, 0.0);
        for (int i : nttm) {
            if (e != cudaSuccess) break;
            const int j = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
            load[j] += work(i);
            hmv_plan_s *p = B->plans[i];
            p->stream = B->side[j];
            const int64_t before = p->launches_total;
            for (int r = 0; r < p->nrhs && e == cudaSuccess; ++r)
                e = ntt_vector_product(p, p->x_limbs_d + static_cast<size_t>(r) * p->n * p->L32,
                                       p->x_neg_d + static_cast<size_t>(r) * p->n, r);
            if (e == cudaSuccess)
                e = launch_round(p, p->n * p->nrhs, p->e_h + p->batch_x_exponent, p->y_limbs_d, p->y_neg_d);
            kernels += p->launches_total - before;  // the rounding's two launches included
            p->stream = B->stream;
        }
        // every branch joins back (also after an error: the capture must end joined)
        for (int j = 0; j < nb; ++j) {
            const cudaError_t je = cudaEventRecord(B->join_ev[j], B->side[j]);
            const cudaError_t we = je == cudaSuccess ? cudaStreamWaitEvent(B->stream, B->join_ev[j], 0) : je;
            if (e == cudaSuccess) e = we;
        }
    }
    // split members: a round per right-hand side
    for (int r = 0; r < B->split_rounds && e == cudaSuccess; ++r) {
        for (size_t i = 0; i < B->plans.size() && e == cudaSuccess; ++i) {
            hmv_plan_s *p = B->plans[i];
            if (!B->split[i] || r >= p->nrhs) continue;
            const int64_t before = p->launches_total;
            e = split_vector_side(p, p->x_limbs_d + static_cast<size_t>(r) * p->n * p->L32,
                                  p->x_neg_d + static_cast<size_t>(r) * p->n);
            kernels += p->launches_total - before;
        }
        for (const auto &sl : B->split_launches) {
            if (sl.round != r || e != cudaSuccess) continue;
            e = launch_leaf_tc_multi(sl.probs, sl.tiles, sl.ntiles, B->split_first->dstat, B->split_first->d_counter,
                                     B->stream, B->num_sms, sl.tn);
            ++kernels;
        }
        for (size_t i = 0; i < B->plans.size() && e == cudaSuccess; ++i) {
            hmv_plan_s *p = B->plans[i];
            if (!B->split[i] || r >= p->nrhs) continue;
            const int64_t before = p->launches_total;
            e = split_post(p, r);
            kernels += p->launches_total - before;
        }
    }
    for (size_t i = 0; i < B->plans.size(); ++i) {
        hmv_plan_s *p = B->plans[i];
        if (B->ntt[i]) continue;  // rounded in its branch
        if (e == cudaSuccess)
            e = launch_round(p, p->n * p->nrhs, p->e_h + p->batch_x_exponent, p->y_limbs_d, p->y_neg_d);
        kernels += 2;
    }
    B->kernels_per_launch = kernels;
    return e;
}

}  // namespace
}  // namespace hmv

using namespace hmv;

extern "C" {

void hmv_batch_free(hmv_batch_t *B) {
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    for (size_t i = 0; i < B->plans.size(); ++i) {
        hmv_plan_s *p = B->plans[i];
        if ((i < B->split.size() && B->split[i]) || (i < B->ntt.size() && B->ntt[i])) {
            hmv_free(p);  // a split or NTT member owns all its buffers
            continue;
        }
        // the batch owns the shared buffers these point to
        p->x_lvl[0] = p->x_lvl[1] = nullptr;
        p->a_lvl[0] = p->a_lvl[1] = nullptr;
        p->post[0] = p->post[1] = nullptr;
        p->xg = nullptr;
        p->leaf_dig = nullptr;
        p->leaf_carry = nullptr;
        hmv_free(p);
    }
    for (void *a : B->allocations) cudaFree(a);
    for (cudaStream_t st : B->side) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : B->join_ev) cudaEventDestroy(ev);
    if (B->fork_ev) cudaEventDestroy(B->fork_ev);
    if (B->own_stream) cudaStreamDestroy(B->stream);
    delete B;
}

hmv_status hmv_batch_create(int32_t count, const hmv_desc *descs, void *stream, uint64_t wave_bytes,
                            hmv_batch_t **out) {
    if (count < 1 || !descs || !out) return HMV_EINVAL;
    for (int i = 0; i < count; ++i) {
        const hmv_desc &d = descs[i];
        if (d.method != HMV_AUTO && d.method != HMV_KARATSUBA && d.method != HMV_NTT) return HMV_EUNSUPPORTED;
        if (d.flags & HMV_FLAG_SIMT_LEAF) return HMV_EUNSUPPORTED;
    }
    hmv_batch_s *B = new (std::nothrow) hmv_batch_s();
    if (!B) return HMV_ENOMEM;
    B->stream = static_cast<cudaStream_t>(stream);
    if (!B->stream) {  // the legacy default stream cannot be captured into a graph
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete B;
            return HMV_ECUDA;
        }
        B->own_stream = true;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        hmv_batch_free(B);
        return HMV_ECUDA;
    }
    const uint32_t kSplitFlags =
        HMV_FLAG_DIGIT_SPLIT1 | HMV_FLAG_DIGIT_SPLIT2 | HMV_FLAG_DIGIT_TOOM4 | HMV_FLAG_DIGIT_TOOM6 | HMV_FLAG_DIGIT_TOOM8;
    for (int i = 0; i < count; ++i) {
        hmv_desc d = descs[i];
        d.flags &= ~HMV_FLAG_TIMING;  // no host-side event syncs inside a graph
        if (d.method == HMV_NTT) {
            hmv_plan_s *p = nullptr;
            const hmv_status st = plan_create(&d, B->stream, false, &p);
            if (st != HMV_OK) { hmv_batch_free(B); return st; }
            B->plans.push_back(p);
            B->split.push_back(0);
            B->ntt.push_back(1);
            continue;
        }
        // split the mantissas where a single HMV_AUTO plan would (or the flags ask)
        bool split = (d.flags & kSplitFlags) != 0;
        if (!split && d.method == HMV_AUTO && d.levels < 0) {
            const int fixed = (d.flags & HMV_FLAG_TILE128) ? 128 : ((d.flags & HMV_FLAG_TILE256) ? 256 : 0);
            split = choose_digit_split(d.n, d.b, B->num_sms, fixed) != 0;
        }
        hmv_plan_s *p = nullptr;
        hmv_status st = plan_create(&d, B->stream, !split, &p);
        if (st == HMV_OK && split && p->children.empty()) {  // not split after all: join the waves
            hmv_free(p);
            p = nullptr;
            split = false;
            st = plan_create(&d, B->stream, true, &p);
        }
        if (st != HMV_OK) { hmv_batch_free(B); return st; }
        B->plans.push_back(p);
        B->split.push_back(split ? 1 : 0);
        B->ntt.push_back(0);
        if (split) {
            B->split_rounds = std::max(B->split_rounds, p->nrhs);
            if (!B->split_first) B->split_first = p;
        }
    }
    cudaError_t e = cudaSuccess;
    int n_ntt = 0;
    for (int i = 0; i < count; ++i) n_ntt += B->ntt[i];
    if (n_ntt > 0) {  // the NTT members' graph branches (kNttBranches at most)
        const int nb = std::min(n_ntt, kNttBranches);
        e = cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming);
        for (int j = 0; j < nb && e == cudaSuccess; ++j) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) B->side.push_back(st);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) B->join_ev.push_back(ev);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            hmv_batch_free(B);
            return HMV_ECUDA;
        }
    }
    size_t mA = 0, mX = 0, mP = 0;
    for (int i = 0; i < count; ++i) {
        if (B->split[i] || B->ntt[i]) continue;
        const hmv_plan_s *p = B->plans[i];
        mA = std::max(mA, p->bytes_a_lvl);
        mX = std::max(mX, p->bytes_x_lvl);
        mP = std::max(mP, p->bytes_post);
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = balloc(B, reinterpret_cast<void **>(&B->a_lvl[k]), mA);
        if (e == cudaSuccess) e = balloc(B, reinterpret_cast<void **>(&B->x_lvl[k]), mX);
        if (e == cudaSuccess) e = balloc(B, reinterpret_cast<void **>(&B->post[k]), mP);
    }
    // waves: the pairs of each leaf tile width in order (one leaf launch per
    // wave, so one width per wave), a new wave when the budget would be exceeded
    std::vector<size_t> wave_size;
    for (int i = 0; i < count; ++i) {
        if (B->split[i] || B->ntt[i]) continue;
        B->plans[i]->a_lvl[0] = B->a_lvl[0];
        B->plans[i]->a_lvl[1] = B->a_lvl[1];
    }
    for (int tn : {256, 128}) {
        bool fresh = true;
        for (int i = 0; i < count; ++i) {
            hmv_plan_s *p = B->plans[i];
            if (B->split[i] || B->ntt[i] || p->tn != tn) continue;
            for (int r = 0; r < p->nrhs; ++r) {
                const size_t sz = pair_bytes(p);
                if (fresh || (wave_size.back() + sz > wave_bytes && wave_size.back() > 0)) {
                    wave_size.push_back(0);
                    B->wave_tn.push_back(tn);
                    fresh = false;
                }
                B->pairs.push_back(Pair{i, r, static_cast<int>(wave_size.size()) - 1, nullptr, nullptr, nullptr});
                wave_size.back() += sz;
            }
        }
    }
    B->nwaves = static_cast<int>(wave_size.size());
    if (!B->pairs.empty()) B->wave_first = B->plans[B->pairs.front().plan];
    const size_t arena_bytes = wave_size.empty() ? 0 : *std::max_element(wave_size.begin(), wave_size.end());
    uint8_t *arena = nullptr;
    if (e == cudaSuccess) e = balloc(B, reinterpret_cast<void **>(&arena), arena_bytes);
    // carve each wave's pairs out of the arena (waves reuse it in turn)
    std::vector<size_t> off(B->nwaves, 0);
    for (Pair &pr : B->pairs) {
        hmv_plan_s *p = B->plans[pr.plan];
        uint8_t *base = arena + off[pr.wave];
        pr.xg = reinterpret_cast<uint16_t *>(base);
        base += align256(p->elems_xg * 2);
        pr.dig = base;
        base += align256(p->bytes_dig);
        pr.carry = reinterpret_cast<int32_t *>(base);
        off[pr.wave] += pair_bytes(p);
    }
    // per wave: leaf problems (own TMA descriptors) and the combined tile list
    for (int w = 0; w < B->nwaves && e == cudaSuccess; ++w) {
        std::vector<LeafProblem> probs;
        std::vector<Tile> tiles;
        for (const Pair &pr : B->pairs) {
            if (pr.wave != w) continue;
            hmv_plan_s *p = B->plans[pr.plan];
            LeafProblem lp;
            memset(&lp, 0, sizeof lp);
            e = encode_tensor_map_A(p, &lp.mapA);
            if (e == cudaSuccess) e = encode_tensor_map_B(p, pr.xg, &lp.mapB);
            if (e != cudaSuccess) break;
            bind(B, p, pr);
            fill_leaf_problem(p, lp);
            const int idx = static_cast<int>(probs.size());
            probs.push_back(lp);
            for (Tile t : p->tiles) {
                t.prob = idx;
                tiles.push_back(t);
            }
            B->leaf_macs += p->leaf_macs;
        }
        if (e != cudaSuccess) break;
        LeafProblem *dp = nullptr;
        Tile *dt = nullptr;
        e = balloc(B, reinterpret_cast<void **>(&dp), probs.size() * sizeof(LeafProblem));
        if (e == cudaSuccess) e = cudaMemcpy(dp, probs.data(), probs.size() * sizeof(LeafProblem), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = balloc(B, reinterpret_cast<void **>(&dt), tiles.size() * sizeof(Tile));
        if (e == cudaSuccess) e = cudaMemcpy(dt, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
        B->d_probs.push_back(dp);
        B->d_tiles.push_back(dt);
        B->ntiles.push_back(static_cast<int>(tiles.size()));
        B->tiles_total += static_cast<int64_t>(tiles.size());
    }
    // split members: per round and tile width, the leaf problems of every
    // unsplit descendant (their own TMA descriptors and buffers) in one list
    for (int r = 0; r < B->split_rounds && e == cudaSuccess; ++r) {
        for (int tn : {256, 128}) {
            std::vector<LeafProblem> probs;
            std::vector<Tile> tiles;
            for (int i = 0; i < count; ++i) {
                hmv_plan_s *p = B->plans[i];
                if (!B->split[i] || r >= p->nrhs) continue;
                std::vector<hmv_plan_s *> leaves;
                collect_leaf_plans(p, leaves);
                for (hmv_plan_s *c : leaves) {
                    if (c->tn != tn) continue;
                    const int idx = static_cast<int>(probs.size());
                    probs.push_back(c->hprob);
                    for (Tile t : c->tiles) {
                        t.prob = idx;
                        tiles.push_back(t);
                    }
                    B->leaf_macs += c->leaf_macs;
                }
            }
            if (tiles.empty()) continue;
            hmv_batch_s::SplitLaunch sl{r, tn, static_cast<int>(tiles.size()), nullptr, nullptr};
            e = balloc(B, reinterpret_cast<void **>(&sl.probs), probs.size() * sizeof(LeafProblem));
            if (e == cudaSuccess)
                e = cudaMemcpy(sl.probs, probs.data(), probs.size() * sizeof(LeafProblem), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = balloc(B, reinterpret_cast<void **>(&sl.tiles), tiles.size() * sizeof(Tile));
            if (e == cudaSuccess)
                e = cudaMemcpy(sl.tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
            B->split_launches.push_back(sl);
            B->tiles_total += static_cast<int64_t>(tiles.size());
        }
    }
    if (e != cudaSuccess) {
        hmv_status st = (e == cudaErrorMemoryAllocation) ? HMV_ENOMEM : HMV_ECUDA;
        hmv_batch_free(B);
        cudaGetLastError();
        return st;
    }
    *out = B;
    return HMV_OK;
}

hmv_status hmv_batch_load_matrix(hmv_batch_t *B, int32_t index, const hmv_vec *h) {
    if (!B || index < 0 || index >= static_cast<int32_t>(B->plans.size())) return HMV_EINVAL;
    if (B->exec) {  // the captured rounding holds the old matrix exponent
        cudaStreamSynchronize(B->stream);
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    return hmv_load_matrix(B->plans[index], h);
}

hmv_status hmv_batch_matvec(hmv_batch_t *B, const hmv_vec *xs, hmv_vec *ys) {
    if (!B || !xs || !ys) return HMV_EINVAL;
    const int count = static_cast<int>(B->plans.size());
    for (int i = 0; i < count; ++i) {
        hmv_plan_s *p = B->plans[i];
        const hmv_vec &x = xs[i], &y = ys[i];
        if (!p->loaded) return HMV_ENOTLOADED;
        if (x.len != p->n || x.nrhs != p->nrhs || x.b != p->b || !x.limbs || !x.neg || x.reserved ||
            y.len != p->n || y.nrhs != p->nrhs || y.b != p->b || !y.limbs || !y.neg || y.reserved ||
            x.on_device != y.on_device || (x.on_device != 0 && x.on_device != 1))
            return HMV_EINVAL;
    }
    cudaError_t e = leaf_tc_prepare();
    // inputs into the buffers the graph reads
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        hmv_plan_s *p = B->plans[i];
        const size_t rows = static_cast<size_t>(p->n) * p->nrhs;
        const cudaMemcpyKind k = xs[i].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        e = cudaMemcpyAsync(p->x_limbs_d, xs[i].limbs, rows * p->L32 * sizeof(uint32_t), k, B->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->x_neg_d, xs[i].neg, rows, k, B->stream);
        if (p->batch_x_exponent != xs[i].exponent && B->exec) {
            // the exponent is a kernel argument of the captured rounding: capture again
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
        p->batch_x_exponent = xs[i].exponent;
    }
    if (e == cudaSuccess && !B->exec) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ie = issue(B);
            e = cudaStreamEndCapture(B->stream, &graph);
            if (e == cudaSuccess) e = ie;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, B->stream);
    if (e == cudaSuccess) B->graph_launches++;
    std::vector<int32_t> st(8 * count, 0);
    for (int i = 0; i < count && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&st[8 * i], B->plans[i]->dstat, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? HMV_ENOMEM : HMV_ECUDA; }
    for (int i = 0; i < count; ++i) {
        if (st[8 * i] == DEV_BADINPUT) return HMV_EINVAL;
        if (st[8 * i] == DEV_TIMEOUT) return HMV_ETIMEOUT;
        if (st[8 * i] != DEV_OK) return HMV_EINTERNAL;
    }
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        hmv_plan_s *p = B->plans[i];
        const size_t rows = static_cast<size_t>(p->n) * p->nrhs;
        const cudaMemcpyKind k = ys[i].on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        e = cudaMemcpyAsync(ys[i].limbs, p->y_limbs_d, rows * p->L32 * sizeof(uint32_t), k, B->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ys[i].neg, p->y_neg_d, rows, k, B->stream);
        ys[i].exponent = st[8 * i + 3];
        p->matvecs++;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    return e == cudaSuccess ? HMV_OK : HMV_ECUDA;
}

hmv_status hmv_batch_get_info(const hmv_batch_t *B, hmv_batch_info *o) {
    if (!B || !o) return HMV_EINVAL;
    memset(o, 0, sizeof *o);
    o->matrices = static_cast<int32_t>(B->plans.size());
    for (const hmv_plan_s *p : B->plans) o->pairs += p->nrhs;
    o->waves = B->nwaves + static_cast<int32_t>(B->split_launches.size());
    o->leaf_tiles = B->tiles_total;
    o->leaf_macs = B->leaf_macs;
    o->device_bytes = B->device_bytes;
    for (const hmv_plan_s *p : B->plans) o->device_bytes += p->device_bytes;
    o->graph_launches = B->graph_launches;
    o->kernels_per_graph = B->kernels_per_launch;
    return HMV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace hmv {
namespace {
// hmv_matvec_many's staging of a step's problem and tile lists, per device.
struct ManyStaging {
    std::mutex mu;
    GrowBuf dev;
    GrowBuf host{nullptr, 0, true};
};
ManyStaging &many_staging() {
    static ManyStaging st[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    return st[dev];
}
}  // namespace
}  // namespace hmv

// One matvec for each of several independent plans, with every leaf product
// in one persistent tensor-core launch: the step of a continuous-batching
// server, whose set of plans changes from one call to the next.  Plans of
// the exact NTT path take part with their own transforms on the same stream
// (they have no leaf products).
extern "C" hmv_status hmv_matvec_many(int32_t count, hmv_plan_t *const *plans, const hmv_vec *xs, hmv_vec *ys) {
    if (count < 1 || !plans || !xs || !ys) return HMV_EINVAL;
    for (int i = 0; i < count; ++i) {
        hmv_plan_s *p = plans[i];
        if (!p) return HMV_EINVAL;
        for (int k = 0; k < i; ++k)
            if (plans[k] == p) return HMV_EINVAL;  // a plan holds one product at a time
        if ((p->method != HMV_KARATSUBA && p->method != HMV_NTT) || p->external_scratch || p->nrhs != 1)
            return HMV_EUNSUPPORTED;
        if (p->method == HMV_KARATSUBA && p->children.empty() && !p->hrev) return HMV_EUNSUPPORTED;  // CUDA-core leaves
        if (!p->loaded) return HMV_ENOTLOADED;
        const hmv_vec &x = xs[i], &y = ys[i];
        if (x.len != p->n || x.nrhs != 1 || x.b != p->b || !x.limbs || !x.neg || x.reserved ||
            y.len != p->n || y.nrhs != 1 || y.b != p->b || !y.limbs || !y.neg || y.reserved ||
            x.on_device != y.on_device || (x.on_device != 0 && x.on_device != 1))
            return HMV_EINVAL;
    }
    cudaStream_t s = plans[0]->stream;
    std::vector<cudaStream_t> saved(count);
    for (int i = 0; i < count; ++i) {
        saved[i] = plans[i]->stream;
        plans[i]->stream = s;
    }
    cudaError_t e = leaf_tc_prepare();
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        hmv_plan_s *p = plans[i];
        const uint32_t *xl = xs[i].limbs;
        const uint8_t *xn = xs[i].neg;
        if (!xs[i].on_device) {
            e = cudaMemcpyAsync(p->x_limbs_d, xl, static_cast<size_t>(p->n) * p->L32 * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(p->x_neg_d, xn, p->n, cudaMemcpyHostToDevice, s);
            xl = p->x_limbs_d;
            xn = p->x_neg_d;
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(p->dstat, 0, 8 * sizeof(int32_t), s);
        if (e == cudaSuccess) e = launch_validate(p, xl, p->n);
        if (p->method == HMV_NTT) {  // the whole product: transforms, pointwise product, extraction
            if (e == cudaSuccess) e = ntt_vector_product(p, xl, xn, 0);
            p->ntt_matvecs++;
            continue;
        }
        if (!p->children.empty()) {  // digit split: the vector side of every unsplit descendant
            if (e == cudaSuccess) e = split_vector_side(p, xl, xn);
            continue;
        }
        if (e == cudaSuccess) e = launch_encode(p, xl, xn, p->n, 0, p->x_lvl[0]);
        for (int l = 0; l < p->L && e == cudaSuccess; ++l)
            e = launch_prepass(p, l, false, p->x_lvl[l % 2], p->x_lvl[(l + 1) % 2]);
        if (e == cudaSuccess) e = launch_pack_vector(p, p->x_lvl[p->L % 2]);
    }
    std::vector<hmv_plan_s *> leafplans;  // every unsplit plan, split plans contributing their descendants
    for (int i = 0; i < count; ++i)
        if (plans[i]->method == HMV_KARATSUBA) collect_leaf_plans(plans[i], leafplans);
    // one persistent launch per tile width present (normally one); the
    // step's problem and tile lists are staged in pinned host memory and
    // copied into device memory, both the library's (per device, grown on
    // demand, held by this call until its last synchronisation)
    std::vector<LeafProblem> gp[2];
    std::vector<Tile> gt[2];
    size_t off_p[2], off_t[2], total = 0;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    for (int w = 0; w < 2; ++w) {
        const int tn = w == 0 ? 256 : 128;
        for (hmv_plan_s *c : leafplans) {
            if (c->tn != tn) continue;
            const int idx = static_cast<int>(gp[w].size());
            gp[w].push_back(c->hprob);
            for (Tile t : c->tiles) {
                t.prob = idx;
                gt[w].push_back(t);
            }
        }
        off_p[w] = total;
        total += al(gp[w].size() * sizeof(LeafProblem));
        off_t[w] = total;
        total += al(gt[w].size() * sizeof(Tile));
    }
    hmv_plan_s *lead = nullptr;  // the leaf launch's tile counter and status word: a Karatsuba plan's
    for (int i = 0; i < count && !lead; ++i)
        if (plans[i]->method == HMV_KARATSUBA) lead = plans[i];
    ManyStaging &ms = many_staging();
    std::unique_lock<std::mutex> staging_lock(ms.mu);
    if (e == cudaSuccess && total > 0) e = grow(ms.dev, total, s);
    if (e == cudaSuccess && total > 0) e = grow(ms.host, total, s);
    if (e == cudaSuccess && total > 0) {
        char *hb = static_cast<char *>(ms.host.ptr);
        for (int w = 0; w < 2; ++w) {
            memcpy(hb + off_p[w], gp[w].data(), gp[w].size() * sizeof(LeafProblem));
            memcpy(hb + off_t[w], gt[w].data(), gt[w].size() * sizeof(Tile));
        }
        e = cudaMemcpyAsync(ms.dev.ptr, hb, total, cudaMemcpyHostToDevice, s);
    }
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) {
        if (gt[w].empty()) continue;
        char *db = static_cast<char *>(ms.dev.ptr);
        e = launch_leaf_tc_multi(reinterpret_cast<LeafProblem *>(db + off_p[w]), reinterpret_cast<Tile *>(db + off_t[w]),
                                 static_cast<int>(gt[w].size()), lead->dstat, lead->d_counter, s, lead->num_sms,
                                 w == 0 ? 256 : 128);
        lead->launches_leaf++;
    }
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        hmv_plan_s *p = plans[i];
        if (p->method == HMV_NTT) {
            // magnitudes, signs and bit lengths already written by the extraction
        } else if (!p->children.empty()) {
            e = split_post(p, 0);
        } else {
            e = launch_post_group(&p, 1);  // leaf normalise and every post-pass level
            if (e == cudaSuccess) e = launch_final_normalize(p, p->post[0], 0, p->post16 ? 2 : 4);
        }
        uint32_t *yl = ys[i].on_device ? ys[i].limbs : p->y_limbs_d;
        uint8_t *yn = ys[i].on_device ? ys[i].neg : p->y_neg_d;
        if (e == cudaSuccess) e = launch_round(p, p->n, p->e_h + xs[i].exponent, yl, yn);
    }
    std::vector<int32_t> st(8 * count, 0);
    for (int i = 0; i < count && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&st[8 * i], plans[i]->dstat, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    for (int i = 0; i < count; ++i) plans[i]->stream = saved[i];
    if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? HMV_ENOMEM : HMV_ECUDA; }
    // a leaf-kernel timeout is recorded in the status word of the first Karatsuba plan
    for (int i = 0; i < count; ++i) {
        if (st[8 * i] == DEV_BADINPUT) return HMV_EINVAL;
        if (st[8 * i] == DEV_TIMEOUT) return HMV_ETIMEOUT;
        if (st[8 * i] != DEV_OK) return HMV_EINTERNAL;
    }
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        hmv_plan_s *p = plans[i];
        if (!ys[i].on_device) {
            e = cudaMemcpyAsync(ys[i].limbs, p->y_limbs_d, static_cast<size_t>(p->n) * p->L32 * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ys[i].neg, p->y_neg_d, p->n, cudaMemcpyDeviceToHost, s);
        }
        ys[i].exponent = st[8 * i + 3];
        p->matvecs++;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HMV_OK : HMV_ECUDA;
}
