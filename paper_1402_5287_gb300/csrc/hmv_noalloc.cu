// Scratch-free schoolbook product: hmv_schoolbook_noalloc.
//
// For callers that cannot allocate device memory while they run: code that
// sits inside another library's or runtime's memory budget, callers on a
// path where a cudaMalloc would synchronise the device or fail under a
// memory cap, and callers that own no allocator at all.  The call uses
// only the caller's input and output buffers plus one fixed scratch array
// compiled into this library, so it never calls cudaMalloc, cudaFree or
// any allocating routine.
//
// The scratch array below is a file-scope __device__ variable: every GPU
// that loads this library holds HMV_NOALLOC_SCRATCH_BYTES of it until the
// process exits, and every call on a device shares it.
#include <mutex>

#include "hmv_internal.h"

namespace hmv {
cudaError_t launch_schoolbook_raw(const uint32_t *hl, const uint8_t *hn, const uint32_t *xl, const uint8_t *xn, int n,
                                  int L32, int circ, __int128 *colsum, cudaStream_t stream);
cudaError_t launch_colsum_round_raw(const __int128 *colsum, int n, int L32, uint32_t *zmag, uint8_t *zneg,
                                    int32_t *zbits, int ZW, int32_t *dstat, int b, int e_in, int reverse,
                                    uint32_t *y, uint8_t *yneg, cudaStream_t stream);

namespace {

static __device__ __align__(256) unsigned char g_scratch[HMV_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Byte offsets of the pieces of one call inside the scratch array.
struct Layout {
    size_t dstat, colsum, zmag, zneg, zbits, total;
};

Layout layout(int n, int L32) {
    const int ZW = 2 * L32 + 2;
    Layout l;
    l.dstat = 0;
    l.colsum = align256(l.dstat + 16 * sizeof(int32_t));
    l.zmag = align256(l.colsum + static_cast<size_t>(n) * 2 * L32 * sizeof(__int128));
    l.zneg = align256(l.zmag + static_cast<size_t>(n) * ZW * sizeof(uint32_t));
    l.zbits = align256(l.zneg + static_cast<size_t>(n));
    l.total = align256(l.zbits + static_cast<size_t>(n) * sizeof(int32_t));
    return l;
}

__global__ void k_check_bits(const uint32_t *limbs, int rows, int L32, int b, int32_t *dstat) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows) return;
    const int topbits = b - 32 * (L32 - 1);
    if (topbits < 32 && (limbs[static_cast<size_t>(k) * L32 + L32 - 1] >> topbits) != 0)
        set_status(dstat, DEV_BADINPUT);
}

// Device address of g_scratch on the current device, looked up once per
// device, on the first call made with that device current (host code cannot
// use the symbol's name as an address).  A cudaDeviceReset unloads the
// module, so the cached address is not valid after one: the header says so.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace hmv

using namespace hmv;

extern "C" hmv_status hmv_schoolbook_noalloc(int32_t n, int32_t b, int32_t kind, const uint32_t *h_limbs,
                                             const uint8_t *h_neg, int32_t h_exponent, const uint32_t *x_limbs,
                                             const uint8_t *x_neg, int32_t x_exponent, uint32_t *y_limbs,
                                             uint8_t *y_neg, int32_t *y_exponent, void *stream) {
    if (n < 1 || b < 1 || b > (1 << 20) || kind < HMV_HANKEL || kind > HMV_CIRCULANT) return HMV_EINVAL;
    if (!h_limbs || !h_neg || !x_limbs || !x_neg || !y_limbs || !y_neg || !y_exponent) return HMV_EINVAL;
    const int L32 = (b + 31) / 32;
    const Layout l = layout(n, L32);
    if (l.total > HMV_NOALLOC_SCRATCH_BYTES) return HMV_EINVAL;  // beyond the compiled-in scratch
    if (!schoolbook_smem_fits(L32)) return HMV_EINVAL;           // a row's operands exceed shared memory
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the call copies to host memory and synchronises the stream, neither of
    // which a capturing stream allows: refuse before queuing anything
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return HMV_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return HMV_EINVAL;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return HMV_ECUDA;
    unsigned char *s = static_cast<unsigned char *>(base);
    int32_t *dstat = reinterpret_cast<int32_t *>(s + l.dstat);
    const int hlen = (kind == HMV_CIRCULANT) ? n : 2 * n - 1;
    // the status words must start at zero; everything else is fully written
    e = cudaMemsetAsync(dstat, 0, 16 * sizeof(int32_t), st);
    if (e == cudaSuccess) {
        k_check_bits<<<(hlen + 127) / 128, 128, 0, st>>>(h_limbs, hlen, L32, b, dstat);
        k_check_bits<<<(n + 127) / 128, 128, 0, st>>>(x_limbs, n, L32, b, dstat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_schoolbook_raw(h_limbs, h_neg, x_limbs, x_neg, n, L32, kind == HMV_CIRCULANT ? 1 : 0,
                                  reinterpret_cast<__int128 *>(s + l.colsum), st);
    if (e == cudaSuccess)
        e = launch_colsum_round_raw(reinterpret_cast<__int128 *>(s + l.colsum), n, L32,
                                    reinterpret_cast<uint32_t *>(s + l.zmag), s + l.zneg,
                                    reinterpret_cast<int32_t *>(s + l.zbits), 2 * L32 + 2, dstat, b,
                                    h_exponent + x_exponent, kind != HMV_HANKEL ? 1 : 0, y_limbs, y_neg, st);
    int32_t hs[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, dstat, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return HMV_ECUDA;
    if (hs[0] == DEV_BADINPUT) return HMV_EINVAL;
    if (hs[0] != DEV_OK) return HMV_EINTERNAL;
    *y_exponent = hs[3];
    return HMV_OK;
}
