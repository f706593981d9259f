// Internal declarations shared by the CUDA translation units of libhmv.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "../../include/hmv.h"
#include "hmv_leaf.h"

namespace hmv {

struct LevelGeom {
    int nodes = 0;                 // 3^l
    int smax = 0;                  // largest node order at this level
    int rowsA = 0;                 // per-node row stride of the matrix side (>= 2*smax-1)
    int rowsX = 0;                 // per-node row stride of the vector side (>= smax)
    std::vector<int> size;         // node orders
    int *d_size = nullptr;         // device copy of size
};

}  // namespace hmv

namespace hmv {
// Working memory that a call needs beyond the plan's fixed buffers, kept by
// the plan and grown on demand: the first call of a size allocates (and a
// larger one reallocates, which synchronises the device); later calls reuse
// it, so the product, inner-product and update calls of a Krylov loop or a
// serving step allocate nothing.
struct GrowBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    bool pinned = false;  // host memory from cudaMallocHost instead of device memory
};
// Device buffers come from the library's memory pool in the order of stream
// s (see pool_alloc); the previous contents are not kept.
cudaError_t grow(GrowBuf &g, size_t bytes, cudaStream_t s);
void release(GrowBuf &g, cudaStream_t s);
// The library's device memory pool (one per device): allocations in stream
// order that keep freed memory for the next plan instead of returning it to
// the device, so that creating and freeing plans neither maps memory nor
// synchronises the device each time; hmv_trim_memory hands it back.
cudaError_t library_pool(cudaMemPool_t *out);
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t s);
void pool_free(void *ptr, cudaStream_t s);
}  // namespace hmv

struct hmv_plan_s {
    hmv_desc desc;
    cudaStream_t stream = nullptr;
    int n = 0, b = 0, nrhs = 1, kind = 0, method = 0;
    int L = 0;                     // Karatsuba depth
    int L32 = 0;                   // limbs per entry
    int Dl = 0;                    // balanced digits per operand in the tree
    int Dp = 0;                    // padded digit stride (multiple of 16)
    int Uo = 0;                    // leaf output digits covered by tiles (multiple of TN)
    int NUB = 0;                   // leaf output digit blocks
    int Wo = 0;                    // post-pass digit stride (multiple of 4)
    int ZW = 0;                    // limbs of the exact rows (Wo / 4)
    int MT = 0;                    // 128-row tiles per leaf
    int tn = hmv::TN_DEFAULT;           // leaf tile width in product digits (256 or 128)
    bool post16 = false;                // post-pass digits as int16 (depth <= 6), else int32
    std::vector<hmv::LevelGeom> lv;
    bool loaded = false;
    int e_h = 0;                   // exponent of the loaded matrix

    // device buffers
    int8_t *a_lvl[2] = {nullptr, nullptr};   // matrix-side digit planes, ping-pong
    int8_t *a_leaf = nullptr;                // matrix-side leaf digits (int8), resident
    int8_t *x_lvl[2] = {nullptr, nullptr};   // vector-side digit planes, ping-pong
    int8_t *x_leaf = nullptr;                // vector-side leaf digits (int8)
    uint16_t *hrev = nullptr;                // bf16 [leaf][RA][Dp], digits reversed
    uint16_t *xg = nullptr;                  // bf16 [leaf][RX][8][Dp], 8 shifted copies
    int RA = 0, RX = 0;
    uint8_t *leaf_dig = nullptr;             // [leaf][MT*TM][Uo]
    int32_t *leaf_carry = nullptr;           // [leaf][MT*TM][NUB]
    int32_t *post[2] = {nullptr, nullptr};   // [node][rowsX][Wo] per level, ping-pong
    uint32_t *zmag = nullptr;                // [nrhs*n][ZW] exact |Z|
    uint8_t *zneg = nullptr;                 // [nrhs*n]
    int32_t *zbits = nullptr;                // [nrhs*n] bit lengths
    int32_t *dstat = nullptr;                // device status block (see k_round_*)
    hmv::Tile *d_tiles = nullptr;
    int ntiles = 0;
    // schoolbook
    __int128 *colsum = nullptr;              // [n][2*L32]
    // staging for host vectors
    uint32_t *x_limbs_d = nullptr, *y_limbs_d = nullptr;
    uint8_t *x_neg_d = nullptr, *y_neg_d = nullptr, *h_neg_d = nullptr;
    uint32_t *h_limbs_d = nullptr;

    CUtensorMap mapA, mapB;
    bool maps_ok = false;
    hmv::LeafProblem *d_prob = nullptr;      // this plan's leaf problem (one entry)
    int *d_counter = nullptr;                // tile counter of the leaf kernel's dynamic schedule
    bool external_scratch = false;           // level, post and leaf buffers owned by a batch
    std::vector<hmv::Tile> tiles;            // host copy of the tile list
    int batch_x_exponent = 0;                // exponent of the x block last given to a batch
    bool dry_run = false;                    // footprint query: nothing is allocated
    // digit-dimension split of the mantissas: Karatsuba (three child plans,
    // V = V1 2^s + V0) or Toom-4 (seven child plans, V = sum_k V_k 2^(ks))
    std::vector<hmv_plan_s *> children;
    int digit_levels = 0;
    int toom = 0;                            // 4 or 6: Toom-Cook split with 2*toom-1 children
    uint32_t **toom_ptrs = nullptr;          // device tables of the children's limb rows (h, then x)
    uint8_t **toom_neg_ptrs = nullptr;
    int64_t *combined64 = nullptr;           // Toom: [n][Wo] int64 digits of Den * Z
    int split_bits = 0;                      // s
    int32_t *combined = nullptr;             // [n][Wo] exact digit vector of this plan's rows
    uint32_t *h_wrap = nullptr;              // circulant: the wrapped Hankel sequence (2n-1 rows)
    uint8_t *h_wrap_neg = nullptr;
    hmv::LeafProblem *split_probs = nullptr; // leaf problems of all unsplit descendants
    hmv::Tile *split_tiles = nullptr;
    hmv::LeafProblem hprob;                  // host copy of *d_prob
    size_t bytes_a_lvl = 0, bytes_x_lvl = 0, bytes_post = 0, elems_xg = 0, bytes_dig = 0, elems_carry = 0;
    int num_sms = 0;
    int64_t device_bytes = 0;
    std::vector<void *> allocations;         // device memory from the library's pool (pool_free at hmv_free)
    // per-call working memory of hmv_dot and hmv_lincomb, grown on demand
    hmv::GrowBuf dot_buf, lin_buf;

    // exact NTT path (two primes): geometry, the matrix spectrum / N, the
    // vector's work array, twiddle tables
    int ntt_P = 0, ntt_S = 0, ntt_K = 0;
    long long ntt_N = 0;
    uint2 *ntt_a = nullptr, *ntt_x = nullptr;
    uint32_t *ntt_tw = nullptr;
    int64_t ntt_matvecs = 0;

    // split-FP64 FFT path
    int fft_w = 0, fft_P = 0, fft_S = 0, fft_K = 0;
    long long fft_N = 0;
    double2 *fft_a = nullptr;                // spectrum of the matrix sequence
    double2 *fft_x = nullptr;                // work array of the vector side
    double2 *fft_tw = nullptr;               // omega_N^m, m < N/2
    unsigned long long *fft_sumsq = nullptr; // exact sums of squares of the pieces [a, x]
    unsigned long long *fft_maxdist = nullptr;
    double fft_sumsq_a = 0, fft_bound = 0, fft_maxdist_h = 0;
    int64_t fft_matvecs = 0, fft_fallbacks = 0;
    double ms_fft = 0;

    // stats
    bool timing = false;
    cudaEvent_t ev[8];
    double ms_prepass = 0, ms_leaf = 0, ms_post = 0, ms_round = 0, ms_total = 0;
    int64_t launches_leaf = 0, launches_total = 0, matvecs = 0;
    double leaf_macs = 0, leaf_macs_issued = 0;
};

namespace hmv {
// launchers (all asynchronous on plan->stream); return a cudaError_t
cudaError_t launch_encode(hmv_plan_s *p, const uint32_t *limbs, const uint8_t *neg, int rows, int circulant_n,
                          int8_t *out);
cudaError_t launch_prepass(hmv_plan_s *p, int level, bool matrix_side, const int8_t *in, int8_t *out);
cudaError_t launch_pack_matrix(hmv_plan_s *p, const int8_t *leaf_digits);
cudaError_t launch_pack_vector(hmv_plan_s *p, const int8_t *leaf_digits);
hmv_status plan_create(const hmv_desc *desc, void *stream, bool external_scratch, hmv_plan_s **out,
                       bool dry_run = false);
cudaError_t launch_validate(hmv_plan_s *p, const uint32_t *limbs, int rows);
cudaError_t launch_colsum_normalize(hmv_plan_s *p, int rhs);
bool ntt_geometry(int n, int b, int &P, int &S, int &K);
size_t ntt_table_words();  // uint32 words of the plan's twiddle tables (ntt_tw)
cudaError_t ntt_init(hmv_plan_s *p);
cudaError_t ntt_load_matrix(hmv_plan_s *p);
cudaError_t ntt_vector_product(hmv_plan_s *p, const uint32_t *xl, const uint8_t *xn, int rhs);
cudaError_t leaf_tc_prepare();
// the unsplit plans under p (p itself when it is not split)
void collect_leaf_plans(hmv_plan_s *p, std::vector<hmv_plan_s *> &out);
hmv_status split_plan_create(hmv_plan_s *p, const hmv_desc &d, int digit_levels);
// HMV_AUTO's digit split for (n, b): 0 (none), Karatsuba levels 1-2, or 4 / 6
// (Toom-K); fixed_tn = 0 lets the tile width vary with the split
int choose_digit_split(int n, int b, int num_sms, int fixed_tn);
hmv_status toom_plan_create(hmv_plan_s *p, const hmv_desc &d, int K);
hmv_status split_load_matrix(hmv_plan_s *p, const uint32_t *h_limbs, const uint8_t *h_neg);
cudaError_t split_vector_side(hmv_plan_s *p, const uint32_t *xl, const uint8_t *xn);
cudaError_t split_leaf_launch(hmv_plan_s *p);
cudaError_t split_post(hmv_plan_s *p, int rhs);
cudaError_t launch_wrap_circulant(hmv_plan_s *p, const uint32_t *c_limbs, const uint8_t *c_neg);
cudaError_t launch_leaf_tc(hmv_plan_s *p);
cudaError_t launch_leaf_tc_multi(const LeafProblem *probs, const Tile *tiles, int ntiles, int32_t *dstat,
                                 int *tile_counter, cudaStream_t stream, int num_sms, int tn);
cudaError_t encode_tensor_map_A(hmv_plan_s *p, CUtensorMap *map);
cudaError_t encode_tensor_map_B(hmv_plan_s *p, uint16_t *xg, CUtensorMap *map);
void fill_leaf_problem(hmv_plan_s *p, LeafProblem &lp);
cudaError_t launch_leaf_simt(hmv_plan_s *p, const int8_t *a_leaf, const int8_t *x_leaf);
// grouped launches for plans of one geometry (same_geometry): the vector side
// from each plan's staged x to its bf16 copies, and leaf normalise plus the
// post-pass down to each plan's level-0 rows
bool same_geometry(hmv_plan_s *const *ps, int G);
cudaError_t launch_colsum_normalize_cols(const __int128 *colsum, int n, int ncols, uint32_t *zmag, uint8_t *zneg,
                                         int32_t *zbits, int ZW, int32_t *dstat, cudaStream_t stream);
cudaError_t launch_colsum_round_cols(const __int128 *colsum, int n, int ncols, int L32, uint32_t *zmag, uint8_t *zneg,
                                     int32_t *zbits, int ZW, int32_t *dstat, int b, int e_in, uint32_t *y,
                                     uint8_t *yneg, cudaStream_t stream);
cudaError_t launch_vector_side_group(hmv_plan_s *const *ps, int G);
cudaError_t launch_post_group(hmv_plan_s *const *ps, int G);
// digit_bytes: 2 (a plan's post buffers with post16), 4 or 8 (int64 Toom sums);
// track_max: also fold the rows' bit lengths into the plan's maximum
cudaError_t launch_final_normalize(hmv_plan_s *p, const int32_t *in, int rhs, int digit_bytes, bool track_max = true);
cudaError_t launch_schoolbook(hmv_plan_s *p, const uint32_t *x_limbs, const uint8_t *x_neg, int rhs);
bool schoolbook_smem_fits(int L32);
cudaError_t launch_round(hmv_plan_s *p, int rows, int e_in, uint32_t *y_limbs, uint8_t *y_neg);
cudaError_t make_tensor_maps(hmv_plan_s *p);
// FFT path (hmv_fft.cu)
double fft_error_bound(double sumsq_a, double sumsq_x, int K);
void fft_geometry(int n, int b, int w, int &P, int &S, int &K);
double fft_worst_bound(int n, int b, int w, int hlen);
cudaError_t fft_init(hmv_plan_s *p);
cudaError_t fft_load_matrix(hmv_plan_s *p);
cudaError_t fft_vector_pieces(hmv_plan_s *p, const uint32_t *xl, const uint8_t *xn);
cudaError_t fft_vector_product(hmv_plan_s *p, int rhs);
}  // namespace hmv
