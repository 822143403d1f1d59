// blink_image_noalloc: the imaging stage (grid -> dirty image) without any device allocation.
//
// Some callers cannot call cudaMalloc while they image: a real-time instrument pipeline that reserves
// all device memory when an observation starts and must not allocate (or risk running out) while data
// stream in, or a host application whose device memory is owned by another allocator (a framework's
// caching pool) that the library may not bypass.  blink_image draws its twiddle table and its
// column-pass workspace from the context, which allocates on first use; this entry point instead uses
// a fixed scratch array reserved in the library's own static device memory, so a call allocates
// nothing.  The kernels are the same column and row passes blink_image launches.
#include <algorithm>
#include <mutex>

#include "blink_internal.cuh"

namespace blink {

int col_block_width(int N);

namespace {

// Scratch of the allocation-free imaging entry point: the twiddle table followed by the column-pass
// result of as many images as fit.  It lives in the module's static device memory, so every GPU that
// loads the library holds these 16 MiB until the process exits.
constexpr size_t kScratchBytes = (size_t)16 << 20;
// room for the largest table: the side-2048 twiddle set or the 8192 unit roots of the mixed-radix passes
constexpr size_t kTwiddleBytes = ((size_t)(tws_total(2048) > 8192 ? tws_total(2048) : 8192) * sizeof(float2) + 255) / 256 * 256;
__device__ __align__(256) unsigned char g_image_scratch[kScratchBytes];

// Device address of g_image_scratch per device.  In host code the array's name stands for a host-side
// shadow, not for device memory, so the address is looked up with cudaGetSymbolAddress, once per device
// with that device current, and passed to the kernels.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

blink_status scratch_for_current_device(void** out) {
    int dev = -1;
    BLINK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(BLINK_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_image_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(image scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BLINK_OK;
}

}  // namespace

}  // namespace blink

using namespace blink;

extern "C" blink_status blink_image_noalloc(const blink_imaging* imaging, const float* d_grid, int32_t n_images,
                                            const float* d_weight, float* d_img, void* stream) {
    BLINK_TRY(check_imaging(imaging));
    BLINK_TRY(nearest_only(imaging, "blink_image_noalloc"));
    const int N = imaging->n_pix, prec = imaging->precision;
    if (!d_grid || !d_weight || !d_img) return set_error(BLINK_ERR_INVALID_ARG, "d_grid, d_weight or d_img is NULL");
    if (n_images < 0) return set_error(BLINK_ERR_INVALID_ARG, "n_images < 0");
    if (((uintptr_t)d_grid & 7) || ((uintptr_t)d_img & 7))
        return set_error(BLINK_ERR_INVALID_ARG, "d_grid and d_img must be 8-byte aligned");
    const bool fast = fast_side(N);
    const int ldh = N / 2 + col_block_width(N);
    const size_t el = prec == BLINK_PREC_BF16 ? 4 : 8;
    const size_t per_img = fast ? (size_t)N * ldh * el : (size_t)N * mixed_h_row(N) * el;
    const size_t room = kScratchBytes - kTwiddleBytes;
    if (per_img > room)
        return set_error(BLINK_ERR_UNSUPPORTED,
                         "blink_image_noalloc: one image's column-pass result exceeds the 16 MiB static scratch "
                         "(largest power-of-two side: 1024 with FP32 storage, 2048 with BF16 storage)");
    // the set-up runs on every call, a zero-image call included, so that such a call can serve as the
    // warm-up that commits the scratch before memory is reserved or a capture begins
    void* scratch = nullptr;
    BLINK_TRY(scratch_for_current_device(&scratch));
    if (n_images == 0) return BLINK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float2* tw = static_cast<float2*>(scratch);
    void* H = static_cast<unsigned char*>(scratch) + kTwiddleBytes;
    const int wave = (int)std::min<size_t>((size_t)n_images, room / per_img);
    if (!fast) {
        BLINK_TRY(make_unit_roots(tw, N, st));
        MixedIn in;
        in.N = N;
        in.tw = tw;
        for (int w0 = 0; w0 < n_images; w0 += wave) {
            const int nw = std::min(wave, n_images - w0);
            in.grid = reinterpret_cast<const float2*>(d_grid) + (int64_t)w0 * N * (N / 2 + 1);
            BLINK_TRY(launch_mixed(in, 0, prec, nw, H, nullptr, 1, WaveMap{1, 0, w0, nw}, 0, nullptr, st));
            BLINK_TRY(launch_mixed(in, 1, prec, nw, H, d_weight, n_images, WaveMap{1, 0, w0, nw}, 0, d_img, st));
        }
        return BLINK_OK;
    }
    BLINK_TRY(make_twiddles(tw, N, st));
    for (int w0 = 0; w0 < n_images; w0 += wave) {
        const int nw = std::min(wave, n_images - w0);
        BLINK_TRY(launch_colpass_grid(N, prec, tw, reinterpret_cast<const float2*>(d_grid) + (int64_t)w0 * N * (N / 2 + 1),
                                      nw, H, ldh, st));
        BLINK_TRY(launch_rowpass(N, prec, tw, H, ldh, 1, d_weight, n_images, WaveMap{1, 0, w0, nw}, nw, 0, d_img, st));
    }
    return BLINK_OK;
}
