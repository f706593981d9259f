// C ABI of libhmv: plans, matrix loading and the matrix-vector product.
//
// Karatsuba path (Beliakov, arXiv:1402.5287, Sec. 3, Algorithm 1), level
// synchronous: every node of a level is handled by one launch.
//   load:    encode h -> matrix-side steps 4 and 6 for levels 0..L-1 ->
//            bf16 leaf slabs (resident)
//   matvec:  encode x -> vector-side steps 3 and 5 for levels 0..L-1 ->
//            leaf products (tensor cores) -> leaf digit normalisation ->
//            step 8 for levels L-1..0 -> exact rows -> b-bit rounding
// Schoolbook path: one CUDA-core kernel on 32-bit limbs -> the same rounding.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "hmv_internal.h"

namespace hmv {
cudaError_t launch_colsum_normalize(hmv_plan_s *p, int rhs);
size_t leaf_tc_smem_bytes();

namespace {

constexpr int kMaxLevels = 16;
constexpr int kMaxBits = 1 << 20;

struct Guard {  // records the first CUDA error of a sequence of calls
    cudaError_t err = cudaSuccess;
    bool operator()(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
        return err == cudaSuccess;
    }
};

hmv_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return HMV_OK;
    if (e == cudaErrorMemoryAllocation) return HMV_ENOMEM;
    return HMV_ECUDA;
}

int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }
long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

// node orders of every level: children of a node of order s have orders
// m = floor((s+1)/2), m, m1 = ceil((s+1)/2)  (Algorithm 1, step 2)
std::vector<LevelGeom> build_levels(int n, int L) {
    std::vector<LevelGeom> lv(L + 1);
    lv[0].nodes = 1;
    lv[0].size = {n};
    for (int l = 0; l < L; ++l) {
        std::vector<int> &ch = lv[l + 1].size;
        ch.reserve(lv[l].size.size() * 3);
        for (int s : lv[l].size) {
            const int m = (s + 1) / 2, m1 = (s + 2) / 2;
            ch.push_back(m);
            ch.push_back(m);
            ch.push_back(m1);
        }
        lv[l + 1].nodes = static_cast<int>(ch.size());
    }
    for (auto &g : lv) {
        g.smax = *std::max_element(g.size.begin(), g.size.end());
        g.rowsA = 2 * g.smax - 1;
        g.rowsX = g.smax;
    }
    return lv;
}

// SM cycles one 128 x tn x 16 MMA takes inside the leaf kernel (measured at
// n = 8000, b = 33220 under Toom-6: 256-wide tiles issue at 0.96 of the
// tensor pipe's rate, 128-wide ones, with two issuing threads, at 0.92).
inline double mma_cycles(int tn) { return tn == 128 ? 67.0 : 128.0; }

// Node orders of every level as (order, count) pairs: a level holds 3^l nodes
// but only a few distinct orders, so the cost model runs in time independent
// of 3^l (building the node lists of deep levels for every candidate depth
// and split dominated plan creation).
struct OrderHist {
    std::vector<std::pair<int, double>> order;  // distinct orders and their node counts
    int smax = 0;
    double nodes = 0;
};

std::vector<OrderHist> order_hists(int n, int L) {
    std::vector<OrderHist> h(L + 1);
    h[0].order = {{n, 1.0}};
    for (int l = 0; l < L; ++l) {
        std::vector<std::pair<int, double>> &ch = h[l + 1].order;
        auto add = [&ch](int s, double c) {
            for (auto &e : ch)
                if (e.first == s) { e.second += c; return; }
            ch.push_back({s, c});
        };
        for (const auto &e : h[l].order) {
            add((e.first + 1) / 2, 2 * e.second);
            add((e.first + 2) / 2, e.second);
        }
    }
    for (auto &g : h)
        for (const auto &e : g.order) {
            g.smax = std::max(g.smax, e.first);
            g.nodes += e.second;
        }
    return h;
}

// K = 16 MMA groups per j-step that a tile over product digits [u0, u0 + tn)
// issues, summed over its s-blocks (as the leaf kernel decodes them: blocks of
// KS digits from s_min rounded down to 8); 128-wide tiles leave out the
// leading groups of the last block that lie wholly above s_max.
int tile_kgroups(int u0, int Dl, int tn) {
    const int s_min = std::max(0, u0 - (Dl - 1)), s_max = std::min(Dl - 1, u0 + tn - 1);
    if (s_max < s_min) return 0;
    const int s_base = s_min / 8 * 8;
    const int nsb = (s_max - s_base + KS) / KS;
    const int kk0 = (s_base + nsb * KS - 1 - s_max) / 16;
    return nsb * (KS / 16) - (tn == 128 ? kk0 : 0);
}

// Estimated seconds of one matvec at depth L on this GPU (tensor work from
// the tile count, memory work from the bytes the level kernels move); hs
// holds the order histograms of at least L + 1 levels.
double cost_model(const std::vector<OrderHist> &hs, int b, int L, int num_sms, int tn) {
    const int Dl = ceil_div(b + L + 2, 8);
    const long long Dp = round_up(Dl, 16);
    const int Uo = static_cast<int>(round_up(2LL * Dl - 1, tn));
    const int NUB = Uo / tn;
    double ksteps = 0;  // 128 x tn x 16 MMAs
    for (int ub = 0; ub < NUB; ++ub) {
        const int kg = tile_kgroups(ub * tn, Dl, tn);
        for (const auto &e : hs[L].order) ksteps += e.second * static_cast<double>(ceil_div(e.first, TM)) * kg * e.first;
    }
    const double mma_s = ksteps * mma_cycles(tn) / (static_cast<double>(num_sms) * 1.9e9);
    double bytes = 0;
    for (int l = 0; l <= L; ++l) bytes += hs[l].nodes * hs[l].smax * (Dp * 2.0 + (Uo + 8) * 4.0 * 4.0);
    bytes += hs[L].nodes * hs[L].smax * Dp * 16.0 * 2.0;
    return mma_s + bytes / 5.0e12;
}

double cost_model(int n, int b, int L, int num_sms, int tn = TN_DEFAULT) {
    return cost_model(order_hists(n, L), b, L, num_sms, tn);
}

// Cheapest index depth for (n, b) and its estimated seconds (depths stop
// once the leaves have order <= 2).
int best_depth(int n, int b, int num_sms, double *cost, int tn = TN_DEFAULT) {
    const std::vector<OrderHist> hs = order_hists(n, kMaxLevels);
    int L = 0;
    double best = 1e300;
    for (int t = 0; t <= kMaxLevels; ++t) {
        if (t > 0 && hs[t - 1].smax <= 2) break;
        const double c = cost_model(hs, b, t, num_sms, tn);
        if (c < best) { best = c; L = t; }
    }
    if (cost) *cost = best;
    return L;
}

// Digit split for HMV_AUTO: kToom4, kToom6, kToom8 or the number of Karatsuba levels d (3^d
// products of about b/2^d bits, d <= 2), each product at its own best depth,
// plus the level kernels, which scale with the products' total width (n*b
// times 1, 3/2, 9/4 for d = 0, 1, 2 and 7/4 for Toom-4; measured 10.4, 15.2,
// 22.4 ms at n = 8000, b = 33220 for d = 0, 1, 2, about 3.9e-11 s per n*b at
// d = 0; (2K-1)/K for Toom-K).  The leaf estimate of the narrower products is
// scaled by (1 - 0.055 d): measured leaf times fall below the tile-count model
// as the products narrow (Toom-K's products count as d = log2 K).  Each
// scheme is costed at both leaf tile widths; *tn gets the cheaper one.
// Toom-8 is left out where its products would need index depth > 7 (its
// int64 interpolation sums are bounded for depths up to 7).
constexpr int kToom4 = 4, kToom6 = 6, kToom8 = 8;
inline bool is_toom(int dl) { return dl == kToom4 || dl == kToom6 || dl == kToom8; }
inline int toom_grow(int K) { return K == 4 ? 4 : (K == 6 ? 9 : 13); }  // bits of |E_t| above s
// only_scheme >= 0 restricts the choice to that scheme (a split the caller
// fixed), leaving only the tile width to choose.
int auto_digit_scheme(int n, int b, int num_sms, int *tn, int fixed_tn, int only_scheme = -1) {
    int best_d = 0;
    double best = 1e300;
    *tn = fixed_tn ? fixed_tn : TN_DEFAULT;
    for (int w : {256, 128}) {
        if (fixed_tn && w != fixed_tn) continue;
        int bd = b;
        double mult = 1.0;
        for (int d = 0; d <= 2; ++d) {
            double leaf = 0;
            best_depth(n, bd, num_sms, &leaf, w);
            const double t = mult * leaf * (1.0 - 0.055 * d) + 3.9e-11 * n * static_cast<double>(b) * std::pow(1.5, d);
            if (t < best && (only_scheme < 0 || only_scheme == d)) { best = t; best_d = d; *tn = w; }
            bd = 32 * (((bd + 31) / 32 + 1) / 2) + 1;  // the children's width
            mult *= 3.0;
        }
        // Toom-K: 2K-1 products of s + g bits; narrowing counted as d = log2 K
        const int L32 = (b + 31) / 32;
        for (int K : {4, 6, 8}) {
            if (L32 < K || (only_scheme >= 0 && only_scheme != K)) continue;
            double leaf = 0;
            const int L = best_depth(n, 32 * ((L32 + K - 1) / K) + toom_grow(K), num_sms, &leaf, w);
            if (K == 8 && L > 7 && only_scheme != K) continue;
            const double t = (2 * K - 1) * leaf * (1.0 - 0.055 * std::log2(static_cast<double>(K))) +
                             3.9e-11 * n * static_cast<double>(b) * (2.0 * K - 1) / K;
            if (t < best) { best = t; best_d = K; *tn = w; }
        }
    }
    return best_d;
}

template <typename T>
cudaError_t dalloc(hmv_plan_s *p, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    if (p->dry_run) {  // footprint query: count the bytes, allocate nothing
        p->device_bytes += static_cast<int64_t>(count * sizeof(T));
        return cudaSuccess;
    }
    void *v = nullptr;
    cudaError_t e = pool_alloc(&v, count * sizeof(T), p->stream);
    if (e != cudaSuccess) return e;
    p->allocations.push_back(v);
    // usable from every stream and by synchronous copies at once, as cudaMalloc's
    e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return e;
    p->device_bytes += static_cast<int64_t>(count * sizeof(T));
    *ptr = static_cast<T *>(v);
    return cudaSuccess;
}

bool valid_vec(const hmv_vec *v, int len, int nrhs, int b) {
    return v && v->len == len && v->nrhs == nrhs && v->b == b && v->limbs && v->neg &&
           (v->on_device == 0 || v->on_device == 1) && v->reserved == 0;
}

__global__ void k_validate(const uint32_t *limbs, int rows, int L32, int b, int32_t *dstat) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows) return;
    const int topbits = b - 32 * (L32 - 1);
    if (topbits < 32 && (limbs[static_cast<size_t>(k) * L32 + L32 - 1] >> topbits) != 0)
        set_status(dstat, DEV_BADINPUT);
}

// Descendants of a split plan report into the top plan's status word.
void share_status(hmv_plan_s *p, int32_t *dstat) {
    for (hmv_plan_s *c : p->children) {
        c->dstat = dstat;
        share_status(c, dstat);
    }
}

}  // namespace

int choose_digit_split(int n, int b, int num_sms, int fixed_tn) {
    int tn = TN_DEFAULT;
    return auto_digit_scheme(n, b, num_sms, &tn, fixed_tn);
}

cudaError_t launch_validate(hmv_plan_s *p, const uint32_t *limbs, int rows) {
    k_validate<<<ceil_div(rows, 128), 128, 0, p->stream>>>(limbs, rows, p->L32, p->b, p->dstat);
    p->launches_total++;
    return cudaGetLastError();
}

namespace {

void timing_mark(hmv_plan_s *p, int k) {
    if (p->timing) cudaEventRecord(p->ev[k], p->stream);
}

float elapsed(hmv_plan_s *p, int a, int b) {
    float ms = 0;
    cudaEventElapsedTime(&ms, p->ev[a], p->ev[b]);
    return ms;
}

}  // namespace
}  // namespace hmv

using namespace hmv;

extern "C" {

const char *hmv_status_string(hmv_status s) {
    switch (s) {
        case HMV_OK: return "ok";
        case HMV_EINVAL: return "invalid argument";
        case HMV_ENOMEM: return "out of memory";
        case HMV_ECUDA: return "CUDA error";
        case HMV_ETIMEOUT: return "device wait timed out";
        case HMV_ENOTLOADED: return "matrix not loaded";
        case HMV_EFFTBOUND: return "FFT error bound not below 1/2";
        case HMV_EUNSUPPORTED: return "unsupported configuration";
        case HMV_EINTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

int32_t hmv_version(void) { return 100; }

void hmv_free(hmv_plan_t *p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);  // the plan's work is done: its memory goes back to the pool at once
    for (hmv_plan_s *c : p->children) hmv_free(c);
    for (void *a : p->allocations) hmv::pool_free(a, p->stream);
    for (hmv::GrowBuf *g : {&p->dot_buf, &p->lin_buf}) hmv::release(*g, p->stream);
    if (p->timing)
        for (auto &e : p->ev) cudaEventDestroy(e);
    delete p;
}

hmv_status hmv_trim_memory(void) {
    cudaMemPool_t pool = nullptr;
    if (hmv::library_pool(&pool) != cudaSuccess) return HMV_ECUDA;
    cudaDeviceSynchronize();  // frees still pending in some stream's order complete first
    return cudaMemPoolTrimTo(pool, 0) == cudaSuccess ? HMV_OK : HMV_ECUDA;
}

hmv_status hmv_plan(const hmv_desc *desc, void *stream, hmv_plan_t **out) {
    return hmv::plan_create(desc, stream, false, out, false);
}

hmv_status hmv_plan_bytes(const hmv_desc *desc, uint64_t *bytes) {
    if (!bytes) return HMV_EINVAL;
    hmv_plan_s *p = nullptr;
    hmv_status st = hmv::plan_create(desc, nullptr, false, &p, true);
    if (st != HMV_OK) return st;
    *bytes = static_cast<uint64_t>(p->device_bytes);
    delete p;
    return HMV_OK;
}

}  // extern "C"

namespace hmv {

// The current device's pool: created on first use, with a release threshold
// of all its memory (freed memory stays reserved for the next allocation).
cudaError_t library_pool(cudaMemPool_t *out) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        int no = 0;  // reuse only memory whose free has completed: no hidden cross-stream dependencies
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t s) {
    *ptr = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = library_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(ptr, bytes ? bytes : 1, pool, s);
    if (e != cudaSuccess) *ptr = nullptr;
    return e;
}

void pool_free(void *ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync(ptr, s);
}

cudaError_t grow(GrowBuf &g, size_t bytes, cudaStream_t s) {
    if (bytes <= g.bytes) return cudaSuccess;
    // the calls that used the old buffer ended with a synchronisation of s
    release(g, s);
    const size_t want = bytes + bytes / 4;  // some room, so that slowly growing calls do not reallocate each time
    cudaError_t e = g.pinned ? cudaMallocHost(&g.ptr, want) : pool_alloc(&g.ptr, want, s);
    if (e != cudaSuccess) {
        g.ptr = nullptr;
        return e;
    }
    g.bytes = want;
    return cudaSuccess;
}

void release(GrowBuf &g, cudaStream_t s) {
    if (g.ptr) {
        if (g.pinned) cudaFreeHost(g.ptr);
        else pool_free(g.ptr, s);
    }
    g.ptr = nullptr;
    g.bytes = 0;
}

hmv_status plan_create(const hmv_desc *desc, void *stream, bool external_scratch, hmv_plan_s **out,
                       bool dry_run) {
    if (!desc || !out) return HMV_EINVAL;
    const hmv_desc &d = *desc;
    if (d.n < 1 || d.b < 1 || d.b > kMaxBits || d.nrhs < 1) return HMV_EINVAL;
    if (d.kind < HMV_HANKEL || d.kind > HMV_CIRCULANT) return HMV_EINVAL;
    if (d.method < HMV_AUTO || d.method > HMV_NTT) return HMV_EINVAL;
    if (d.levels < -1 || d.levels > kMaxLevels) return HMV_EINVAL;
    if (d.flags & ~(HMV_FLAG_TIMING | HMV_FLAG_SIMT_LEAF | HMV_FLAG_DIGIT_SPLIT1 | HMV_FLAG_DIGIT_SPLIT2 |
                    HMV_FLAG_TILE128 | HMV_FLAG_TILE256 | HMV_FLAG_DIGIT_TOOM4 | HMV_FLAG_DIGIT_TOOM6 |
                    HMV_FLAG_DIGIT_TOOM8))
        return HMV_EINVAL;
    if ((d.flags & HMV_FLAG_TILE128) && (d.flags & HMV_FLAG_TILE256)) return HMV_EINVAL;
    const uint32_t split_flags =
        d.flags & (HMV_FLAG_DIGIT_SPLIT1 | HMV_FLAG_DIGIT_SPLIT2 | HMV_FLAG_DIGIT_TOOM4 | HMV_FLAG_DIGIT_TOOM6 |
                   HMV_FLAG_DIGIT_TOOM8);
    if (split_flags & (split_flags - 1)) return HMV_EINVAL;  // at most one digit split
    int digit_levels = (d.flags & HMV_FLAG_DIGIT_SPLIT2) ? 2 : ((d.flags & HMV_FLAG_DIGIT_SPLIT1) ? 1 : 0);
    if (d.flags & HMV_FLAG_DIGIT_TOOM4) digit_levels = kToom4;
    if (d.flags & HMV_FLAG_DIGIT_TOOM6) digit_levels = kToom6;
    if (d.flags & HMV_FLAG_DIGIT_TOOM8) digit_levels = kToom8;
    if (digit_levels && ((d.method != HMV_AUTO && d.method != HMV_KARATSUBA) || (d.flags & HMV_FLAG_SIMT_LEAF)))
        return HMV_EINVAL;
    if (is_toom(digit_levels) && (d.b + 31) / 32 < digit_levels)
        return HMV_EINVAL;  // K parts of at least one limb
    if (d.method == HMV_FFT64 ? (d.piece_bits != 0 && (d.piece_bits < 4 || d.piece_bits > 16)) : d.piece_bits != 0)
        return HMV_EINVAL;
    if (static_cast<long long>(d.n) * d.nrhs > (1LL << 30)) return HMV_EINVAL;
    if (d.method == HMV_NTT) {
        if (d.levels > 0 || (d.flags & ~HMV_FLAG_TIMING)) return HMV_EINVAL;
        int P, S, K;
        if (!ntt_geometry(d.n, d.b, P, S, K)) return HMV_EUNSUPPORTED;
    }

    hmv_plan_s *p = new (std::nothrow) hmv_plan_s();
    if (!p) return HMV_ENOMEM;
    p->desc = d;
    p->stream = static_cast<cudaStream_t>(stream);
    p->n = d.n;
    p->b = d.b;
    p->nrhs = d.nrhs;
    p->kind = d.kind;
    p->method = (d.method == HMV_AUTO) ? HMV_KARATSUBA : d.method;
    p->L32 = (d.b + 31) / 32;
    p->timing = (d.flags & HMV_FLAG_TIMING) != 0;
    p->external_scratch = external_scratch;
    p->tn = (d.flags & HMV_FLAG_TILE128) ? 128 : TN_DEFAULT;
    if (external_scratch && (p->method != HMV_KARATSUBA || (d.flags & HMV_FLAG_SIMT_LEAF))) {
        delete p;
        return HMV_EUNSUPPORTED;
    }
    p->dry_run = dry_run;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) {
        if (!dry_run) { delete p; return from_cuda(ce); }
        cudaGetLastError();
        p->num_sms = 152;  // footprint query without a device: GB300's SM count
    }
    if (p->method == HMV_SCHOOLBOOK && !dry_run && !schoolbook_smem_fits(p->L32)) {
        delete p;
        return HMV_EINVAL;  // one row's operands do not fit the kernel's shared memory
    }
    if (p->timing && !dry_run)
        for (auto &e : p->ev) cudaEventCreate(&e);
    else
        p->timing = false;

    Guard g;
    const int n = d.n;
    int dl = digit_levels;
    if (d.method == HMV_AUTO && d.levels < 0 && !(d.flags & HMV_FLAG_SIMT_LEAF) && !external_scratch) {
        const bool fixed = (d.flags & (HMV_FLAG_TILE128 | HMV_FLAG_TILE256)) != 0;
        int tn = TN_DEFAULT;
        // the split by the cost model, or the caller's split with the cost model's tile width
        dl = auto_digit_scheme(n, d.b, p->num_sms, &tn, fixed ? p->tn : 0, dl == 0 ? -1 : dl);
        // a split plan's products take the scheme's tile width
        if (dl != 0) p->tn = tn;
    }
    digit_levels = dl;
    const bool toom = is_toom(digit_levels);
    p->digit_levels = toom ? 0 : digit_levels;
    if (digit_levels && !external_scratch) {
        hmv_status st = toom ? toom_plan_create(p, d, digit_levels) : split_plan_create(p, d, digit_levels);
        if (st != HMV_OK) { hmv_free(p); return st; }
        if (toom) g(dalloc(p, &p->combined64, static_cast<size_t>(n) * p->Wo));
        else g(dalloc(p, &p->combined, static_cast<size_t>(n) * p->Wo));
        g(dalloc(p, &p->d_counter, 1));
        if (toom) {
            // the children's staging rows never move: one table for the matrix side, one for x
            const int P = static_cast<int>(p->children.size());
            g(dalloc(p, &p->toom_ptrs, 2 * P));
            g(dalloc(p, &p->toom_neg_ptrs, 2 * P));
            uint32_t *tl[30];
            uint8_t *tn[30];
            for (int t = 0; t < P; ++t) {
                tl[t] = p->children[t]->h_limbs_d;
                tn[t] = p->children[t]->h_neg_d;
                tl[P + t] = p->children[t]->x_limbs_d;
                tn[P + t] = p->children[t]->x_neg_d;
            }
            if (!dry_run && g.err == cudaSuccess) {
                g(cudaMemcpy(p->toom_ptrs, tl, 2 * P * sizeof(uint32_t *), cudaMemcpyHostToDevice));
                g(cudaMemcpy(p->toom_neg_ptrs, tn, 2 * P * sizeof(uint8_t *), cudaMemcpyHostToDevice));
            }
        }
        if (d.kind == HMV_CIRCULANT) {
            g(dalloc(p, &p->h_wrap, static_cast<size_t>(2 * n - 1) * p->L32));
            g(dalloc(p, &p->h_wrap_neg, static_cast<size_t>(2 * n - 1)));
        }
    } else if (p->method == HMV_SCHOOLBOOK) {
        p->L = 0;
        p->ZW = 2 * p->L32 + 2;
        g(dalloc(p, &p->colsum, static_cast<size_t>(n) * 2 * p->L32));
    } else if (p->method == HMV_NTT) {
        p->L = 0;
        p->ZW = 2 * p->L32 + 2;  // |Z| < n 2^(2b)
        ntt_geometry(n, d.b, p->ntt_P, p->ntt_S, p->ntt_K);
        p->ntt_N = 1LL << p->ntt_K;
        g(dalloc(p, &p->ntt_a, static_cast<size_t>(p->ntt_N)));
        g(dalloc(p, &p->ntt_x, static_cast<size_t>(p->ntt_N)));
        g(dalloc(p, &p->ntt_tw, ntt_table_words()));
        if (g.err == cudaSuccess && !dry_run) g(ntt_init(p));
    } else {
        // depth: explicit, or the cheapest by the cost model (node order >= 2);
        // under HMV_AUTO the tile width too (128 only pays where it cuts the
        // padded product digits enough, i.e. for short mantissas)
        int L = d.levels;
        const bool auto_tile =
            d.method == HMV_AUTO && !(d.flags & (HMV_FLAG_TILE128 | HMV_FLAG_TILE256 | HMV_FLAG_SIMT_LEAF));
        if (auto_tile) {
            double c256 = 0, c128 = 0;
            const int L256 = L < 0 ? best_depth(n, d.b, p->num_sms, &c256, 256) : L;
            const int L128 = L < 0 ? best_depth(n, d.b, p->num_sms, &c128, 128) : L;
            if (L >= 0) {
                c256 = cost_model(n, d.b, L, p->num_sms, 256);
                c128 = cost_model(n, d.b, L, p->num_sms, 128);
            }
            p->tn = c128 < c256 ? 128 : 256;
            L = c128 < c256 ? L128 : L256;
        } else if (L < 0) {
            L = best_depth(n, d.b, p->num_sms, nullptr, p->tn);
        }
        p->L = L;
        p->lv = build_levels(n, L);
        p->Dl = ceil_div(static_cast<long long>(d.b) + L + 2, 8);
        p->Dp = static_cast<int>(round_up(p->Dl, 16));
        p->Uo = static_cast<int>(round_up(2LL * p->Dl - 1, p->tn));
        p->NUB = p->Uo / p->tn;
        p->Wo = p->Uo + EXTRA_DIGITS;
        p->ZW = p->Wo / 4;
        const LevelGeom &leaf = p->lv[L];
        p->MT = ceil_div(leaf.smax, TM);
        p->RA = static_cast<int>(round_up(leaf.rowsA, 32));  // whole 32-row groups for the A tensor map
        p->RX = leaf.rowsX;
        size_t maxA = 0, maxX = 0, maxPost = 0;
        for (auto &lg : p->lv) {
            maxA = std::max(maxA, static_cast<size_t>(lg.nodes) * lg.rowsA * p->Dp);
            maxX = std::max(maxX, static_cast<size_t>(lg.nodes) * lg.rowsX * p->Dp);
            maxPost = std::max(maxPost, static_cast<size_t>(lg.nodes) * lg.rowsX * p->Wo);
        }
        for (auto &lg : p->lv) {
            if (dry_run) { p->device_bytes += static_cast<int64_t>(lg.size.size() * sizeof(int)); continue; }
            if (g(dalloc(p, &lg.d_size, lg.size.size())))
                g(cudaMemcpyAsync(lg.d_size, lg.size.data(), lg.size.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  p->stream));
        }
        const bool simt = (d.flags & HMV_FLAG_SIMT_LEAF) != 0;
        p->bytes_a_lvl = maxA;
        p->bytes_x_lvl = maxX;
        // post-pass digits: leaf digits lie in [-128, 510] and each level at most
        // doubles them, so int16 holds them through 6 levels
        p->post16 = L <= 6;
        p->bytes_post = maxPost * (p->post16 ? sizeof(int16_t) : sizeof(int32_t));
        p->elems_xg = static_cast<size_t>(leaf.nodes) * p->RX * 8 * (p->Dp + 8);
        p->bytes_dig = static_cast<size_t>(leaf.nodes) * p->MT * TM * p->Uo;
        p->elems_carry = static_cast<size_t>(leaf.nodes) * p->MT * TM * p->NUB;
        if (!simt) g(dalloc(p, &p->hrev, static_cast<size_t>(leaf.nodes) * p->RA * p->Dp));
        if (!external_scratch) {
            g(dalloc(p, &p->a_lvl[0], maxA));
            if (L > 0) g(dalloc(p, &p->a_lvl[1], maxA));
            g(dalloc(p, &p->x_lvl[0], maxX));
            if (L > 0) g(dalloc(p, &p->x_lvl[1], maxX));
            if (!simt) g(dalloc(p, &p->xg, p->elems_xg));
            g(dalloc(p, &p->leaf_dig, p->bytes_dig));
            g(dalloc(p, &p->leaf_carry, p->elems_carry));
            const size_t post_words = (p->bytes_post + sizeof(int32_t) - 1) / sizeof(int32_t);
            g(dalloc(p, &p->post[0], post_words));
            if (L > 0) g(dalloc(p, &p->post[1], post_words));
        }
        // tiles: leaf-major (neighbouring CTAs share a leaf's operands in L2),
        // within a leaf the longest K loops first
        std::vector<Tile> tiles;
        double macs = 0, issued = 0;
        for (int lf = 0; lf < leaf.nodes; ++lf) {
            const int m = leaf.size[lf];
            std::vector<Tile> lt;
            for (int mt = 0; mt < ceil_div(m, TM); ++mt)
                for (int ub = 0; ub < p->NUB; ++ub) {
                    const int kg = tile_kgroups(ub * p->tn, p->Dl, p->tn);  // as the kernel
                    lt.push_back(Tile{lf, mt * TM, ub, kg * m, 0});
                    issued += static_cast<double>(TM) * p->tn * 16 * kg * m;
                }
            std::stable_sort(lt.begin(), lt.end(), [](const Tile &a, const Tile &b2) { return a.cost > b2.cost; });
            tiles.insert(tiles.end(), lt.begin(), lt.end());
            macs += static_cast<double>(m) * m * static_cast<double>(p->Dl) * p->Dl;
        }
        p->leaf_macs = macs;
        p->leaf_macs_issued = issued;
        p->ntiles = static_cast<int>(tiles.size());
        p->tiles = tiles;
        if (g(dalloc(p, &p->d_tiles, tiles.size())) && !dry_run)
            g(cudaMemcpy(p->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
        if (!simt) g(dalloc(p, &p->d_prob, 1));
        if (!simt) g(dalloc(p, &p->d_counter, 1));
        if (!simt && !external_scratch && !dry_run && g.err == cudaSuccess) g(make_tensor_maps(p));
    }
    const int hlen0 = (d.kind == HMV_CIRCULANT) ? n : 2 * n - 1;
    if (p->method == HMV_FFT64) {
        int w = d.piece_bits;
        if (w == 0) {  // the largest width whose worst-case bound is below 1/2
            w = 4;
            for (int t = 16; t >= 4; --t)
                if (fft_worst_bound(n, d.b, t, hlen0) < 0.5) { w = t; break; }
        }
        p->fft_w = w;
        fft_geometry(n, d.b, w, p->fft_P, p->fft_S, p->fft_K);
        p->fft_N = 1LL << p->fft_K;
        p->ZW = std::max(p->ZW, ceil_div(static_cast<long long>(w) * (2 * p->fft_P + 3), 32) + 1);
        g(dalloc(p, &p->fft_a, static_cast<size_t>(p->fft_N)));
        g(dalloc(p, &p->fft_x, static_cast<size_t>(p->fft_N)));
        g(dalloc(p, &p->fft_tw, static_cast<size_t>(p->fft_N / 2)));
        g(dalloc(p, &p->fft_sumsq, 2));
        g(dalloc(p, &p->fft_maxdist, 1));
        if (g.err == cudaSuccess && !dry_run) g(fft_init(p));
    }
    const int hlen = (d.kind == HMV_CIRCULANT) ? n : 2 * n - 1;
    const size_t rows = static_cast<size_t>(n) * d.nrhs;
    g(dalloc(p, &p->zmag, rows * p->ZW));
    g(dalloc(p, &p->zneg, rows));
    g(dalloc(p, &p->zbits, rows));
    g(dalloc(p, &p->dstat, 8));
    g(dalloc(p, &p->x_limbs_d, rows * p->L32));
    g(dalloc(p, &p->x_neg_d, rows));
    g(dalloc(p, &p->y_limbs_d, rows * p->L32));
    g(dalloc(p, &p->y_neg_d, rows));
    g(dalloc(p, &p->h_limbs_d, static_cast<size_t>(hlen) * p->L32));
    g(dalloc(p, &p->h_neg_d, hlen));
    if (g.err != cudaSuccess) {
        hmv_status st = from_cuda(g.err);
        hmv_free(p);
        cudaGetLastError();
        return st;
    }
    if (!p->children.empty()) share_status(p, p->dstat);
    // the pool's allocations (and the copies above) are complete: every
    // stream may use the plan's memory from now on
    if (!dry_run && !g(cudaStreamSynchronize(p->stream))) {
        hmv_status st = from_cuda(g.err);
        hmv_free(p);
        cudaGetLastError();
        return st;
    }
    *out = p;
    return HMV_OK;
}

}  // namespace hmv

extern "C" {

hmv_status hmv_load_matrix(hmv_plan_t *p, const hmv_vec *h) {
    if (!p) return HMV_EINVAL;
    const int hlen = (p->kind == HMV_CIRCULANT) ? p->n : 2 * p->n - 1;
    if (!valid_vec(h, hlen, 1, p->b)) return HMV_EINVAL;
    p->loaded = false;
    Guard g;
    const size_t nl = static_cast<size_t>(hlen) * p->L32;
    const cudaMemcpyKind kind = h->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (h->limbs != p->h_limbs_d)  // a split parent may hand a child its own staging buffer
        g(cudaMemcpyAsync(p->h_limbs_d, h->limbs, nl * sizeof(uint32_t), kind, p->stream));
    if (h->neg != p->h_neg_d) g(cudaMemcpyAsync(p->h_neg_d, h->neg, hlen, kind, p->stream));
    g(cudaMemsetAsync(p->dstat, 0, 8 * sizeof(int32_t), p->stream));
    k_validate<<<ceil_div(hlen, 128), 128, 0, p->stream>>>(p->h_limbs_d, hlen, p->L32, p->b, p->dstat);
    g(cudaGetLastError());
    if (!p->children.empty()) {
        int32_t vs[8] = {0};
        g(cudaMemcpyAsync(vs, p->dstat, sizeof vs, cudaMemcpyDeviceToHost, p->stream));
        g(cudaStreamSynchronize(p->stream));
        if (g.err != cudaSuccess) return from_cuda(g.err);
        if (vs[0] == DEV_BADINPUT) return HMV_EINVAL;
        const uint32_t *hl = p->h_limbs_d;
        const uint8_t *hn = p->h_neg_d;
        if (p->kind == HMV_CIRCULANT) {
            g(launch_wrap_circulant(p, p->h_limbs_d, p->h_neg_d));
            hl = p->h_wrap;
            hn = p->h_wrap_neg;
        }
        if (g.err != cudaSuccess) return from_cuda(g.err);
        hmv_status st = split_load_matrix(p, hl, hn);
        if (st != HMV_OK) return st;
        p->e_h = h->exponent;
        p->loaded = true;
        return HMV_OK;
    }
    if (p->method != HMV_SCHOOLBOOK && p->method != HMV_NTT) {
        // level 0 holds the Hankel sequence (circulant: the wrapped Toeplitz sequence)
        g(launch_encode(p, p->h_limbs_d, p->h_neg_d, 2 * p->n - 1, p->kind == HMV_CIRCULANT ? p->n : 0, p->a_lvl[0]));
        for (int l = 0; l < p->L; ++l) g(launch_prepass(p, l, true, p->a_lvl[l % 2], p->a_lvl[(l + 1) % 2]));
        p->a_leaf = p->a_lvl[p->L % 2];
        if (p->hrev) g(launch_pack_matrix(p, p->a_leaf));
    }
    if (p->method == HMV_FFT64) g(fft_load_matrix(p));
    if (p->method == HMV_NTT) g(ntt_load_matrix(p));
    int32_t st[8] = {0};
    g(cudaMemcpyAsync(st, p->dstat, sizeof st, cudaMemcpyDeviceToHost, p->stream));
    g(cudaStreamSynchronize(p->stream));
    if (g.err != cudaSuccess) return from_cuda(g.err);
    if (st[0] == DEV_BADINPUT) return HMV_EINVAL;
    if (st[0] != DEV_OK) return HMV_EINTERNAL;
    if (p->method == HMV_FFT64) {
        unsigned long long sq = 0;
        if (!g(cudaMemcpy(&sq, p->fft_sumsq, sizeof sq, cudaMemcpyDeviceToHost))) return from_cuda(g.err);
        p->fft_sumsq_a = static_cast<double>(sq);
    }
    p->e_h = h->exponent;
    p->loaded = true;
    return HMV_OK;
}

hmv_status hmv_matvec(hmv_plan_t *p, const hmv_vec *x, hmv_vec *y) {
    if (!p) return HMV_EINVAL;
    if (!valid_vec(x, p->n, p->nrhs, p->b) || !valid_vec(y, p->n, p->nrhs, p->b)) return HMV_EINVAL;
    if (x->on_device != y->on_device) return HMV_EINVAL;
    if (!p->loaded) return HMV_ENOTLOADED;
    Guard g;
    const size_t rows = static_cast<size_t>(p->n) * p->nrhs;
    const uint32_t *xl = x->limbs;
    const uint8_t *xn = x->neg;
    timing_mark(p, 0);
    if (!x->on_device) {
        g(cudaMemcpyAsync(p->x_limbs_d, x->limbs, rows * p->L32 * sizeof(uint32_t), cudaMemcpyHostToDevice,
                          p->stream));
        g(cudaMemcpyAsync(p->x_neg_d, x->neg, rows, cudaMemcpyHostToDevice, p->stream));
        xl = p->x_limbs_d;
        xn = p->x_neg_d;
    }
    g(cudaMemsetAsync(p->dstat, 0, 8 * sizeof(int32_t), p->stream));
    k_validate<<<ceil_div(static_cast<long long>(rows), 128), 128, 0, p->stream>>>(xl, static_cast<int>(rows), p->L32,
                                                                                  p->b, p->dstat);
    g(cudaGetLastError());
    timing_mark(p, 1);
    float ms_pre = 0, ms_leaf = 0, ms_post = 0;
    for (int r = 0; r < p->nrhs && g.err == cudaSuccess; ++r) {
        const uint32_t *xr = xl + static_cast<size_t>(r) * p->n * p->L32;
        const uint8_t *xnr = xn + static_cast<size_t>(r) * p->n;
        bool use_fft = false;
        if (p->method == HMV_FFT64) {
            // the bound needs the exact norm of this vector's pieces
            g(fft_vector_pieces(p, xr, xnr));
            unsigned long long sq = 0;
            g(cudaMemcpyAsync(&sq, p->fft_sumsq + 1, sizeof sq, cudaMemcpyDeviceToHost, p->stream));
            g(cudaStreamSynchronize(p->stream));
            p->fft_bound = fft_error_bound(p->fft_sumsq_a, static_cast<double>(sq), p->fft_K);
            use_fft = p->fft_bound < 0.5;
            if (use_fft) p->fft_matvecs++;
            else p->fft_fallbacks++;
        }
        if (!p->children.empty()) {
            g(split_vector_side(p, xr, xnr));
            timing_mark(p, 2);
            g(split_leaf_launch(p));
            timing_mark(p, 3);
            g(split_post(p, r));
            timing_mark(p, 4);
        } else if (use_fft) {
            timing_mark(p, 2);
            g(cudaMemsetAsync(p->fft_maxdist, 0, sizeof(unsigned long long), p->stream));
            g(fft_vector_product(p, r));
            timing_mark(p, 3);
            timing_mark(p, 4);
        } else if (p->method == HMV_NTT) {
            timing_mark(p, 2);
            g(ntt_vector_product(p, xr, xnr, r));
            p->ntt_matvecs++;
            timing_mark(p, 3);
            timing_mark(p, 4);
        } else if (p->method == HMV_SCHOOLBOOK) {
            timing_mark(p, 2);
            g(launch_schoolbook(p, xr, xnr, r));
            timing_mark(p, 3);
            g(launch_colsum_normalize(p, r));
            timing_mark(p, 4);
        } else {
            g(launch_encode(p, xr, xnr, p->n, 0, p->x_lvl[0]));
            for (int l = 0; l < p->L; ++l) g(launch_prepass(p, l, false, p->x_lvl[l % 2], p->x_lvl[(l + 1) % 2]));
            const int8_t *x_leaf = p->x_lvl[p->L % 2];
            if (p->xg) g(launch_pack_vector(p, x_leaf));
            timing_mark(p, 2);
            if (p->xg) g(launch_leaf_tc(p));
            else g(launch_leaf_simt(p, p->a_leaf, x_leaf));
            timing_mark(p, 3);
            g(launch_post_group(&p, 1));  // leaf normalise and every post-pass level
            g(launch_final_normalize(p, p->post[0], r, p->post16 ? 2 : 4));
            timing_mark(p, 4);
        }
        if (p->timing && g.err == cudaSuccess) {
            g(cudaEventSynchronize(p->ev[4]));
            ms_pre += elapsed(p, 1, 2);
            if (use_fft) p->ms_fft += elapsed(p, 2, 3);
            else ms_leaf += elapsed(p, 2, 3);
            ms_post += elapsed(p, 3, 4);
        }
        timing_mark(p, 1);
    }
    uint32_t *yl = y->on_device ? y->limbs : p->y_limbs_d;
    uint8_t *yn = y->on_device ? y->neg : p->y_neg_d;
    timing_mark(p, 5);
    g(launch_round(p, static_cast<int>(rows), p->e_h + x->exponent, yl, yn));
    timing_mark(p, 6);
    int32_t st[8] = {0};
    g(cudaMemcpyAsync(st, p->dstat, sizeof st, cudaMemcpyDeviceToHost, p->stream));
    g(cudaStreamSynchronize(p->stream));
    if (g.err != cudaSuccess) return from_cuda(g.err);
    if (st[0] == DEV_BADINPUT) return HMV_EINVAL;
    if (st[0] == DEV_TIMEOUT) return HMV_ETIMEOUT;
    if (st[0] != DEV_OK) return HMV_EINTERNAL;
    if (!y->on_device) {
        g(cudaMemcpyAsync(y->limbs, yl, rows * p->L32 * sizeof(uint32_t), cudaMemcpyDeviceToHost, p->stream));
        g(cudaMemcpyAsync(y->neg, yn, rows, cudaMemcpyDeviceToHost, p->stream));
        g(cudaStreamSynchronize(p->stream));
        if (g.err != cudaSuccess) return from_cuda(g.err);
    }
    y->exponent = st[3];
    if (p->method == HMV_FFT64) {
        unsigned long long md = 0;
        if (!g(cudaMemcpy(&md, p->fft_maxdist, sizeof md, cudaMemcpyDeviceToHost))) return from_cuda(g.err);
        double dd;
        memcpy(&dd, &md, sizeof dd);
        p->fft_maxdist_h = dd;
    }
    if (p->timing) {
        p->ms_prepass += ms_pre;
        p->ms_leaf += ms_leaf;
        p->ms_post += ms_post;
        p->ms_round += elapsed(p, 5, 6);
        p->ms_total += elapsed(p, 0, 6);
    }
    p->matvecs++;
    return HMV_OK;
}

hmv_status hmv_get_stats(const hmv_plan_t *p, hmv_stats *o) {
    if (!p || !o) return HMV_EINVAL;
    memset(o, 0, sizeof *o);
    const hmv_plan_s *q = p;
    int unsplit = 1;
    while (!q->children.empty()) {
        unsplit *= static_cast<int>(q->children.size());
        q = q->children[0];
    }
    o->levels = q->L;
    o->leaves = unsplit * (q->lv.empty() ? 1 : q->lv[q->L].nodes);
    o->leaf_rows_max = q->lv.empty() ? q->n : q->lv[q->L].smax;
    o->digits = q->Dl;
    o->leaf_tiles = p->ntiles;
    o->leaf_macs = p->leaf_macs;
    o->leaf_macs_issued = p->leaf_macs_issued;
    o->device_bytes = p->device_bytes;
    o->ms_prepass = p->ms_prepass;
    o->ms_leaf = p->ms_leaf;
    o->ms_post = p->ms_post;
    o->ms_round = p->ms_round;
    o->ms_total = p->ms_total;
    o->launches_leaf = p->launches_leaf;
    o->launches_total = p->launches_total;
    o->matvecs = p->matvecs;
    o->fft_piece_bits = p->method == HMV_NTT ? 16 : p->fft_w;
    o->fft_log2_len = p->method == HMV_NTT ? p->ntt_K : p->fft_K;
    o->fft_bound = p->fft_bound;
    o->fft_max_dist = p->fft_maxdist_h;
    o->fft_matvecs = p->fft_matvecs;
    o->fft_fallbacks = p->fft_fallbacks;
    o->ms_fft = p->ms_fft;
    o->leaf_tile_digits = (q->method == HMV_KARATSUBA && !q->lv.empty() && q->hrev) ? q->tn : 0;
    o->digit_products = unsplit;
    return HMV_OK;
}

hmv_status hmv_reset_stats(hmv_plan_t *p) {
    if (!p) return HMV_EINVAL;
    p->ms_prepass = p->ms_leaf = p->ms_post = p->ms_round = p->ms_total = p->ms_fft = 0;
    p->launches_leaf = p->launches_total = p->matvecs = 0;
    p->fft_matvecs = p->fft_fallbacks = 0;
    return HMV_OK;
}

}  // extern "C"
