// ft_noalloc.cu -- ft_topk_per_band_noalloc: the candidate search with no device allocation.
//
// ft_topk_per_band keeps its per-CTA candidate lists in context scratch that it grows with
// cudaMalloc on demand.  Some callers cannot let a library allocate: a process whose device
// memory is already reserved by another allocator (a framework's caching allocator or a
// fixed memory budget set at start-up, where a fresh cudaMalloc can fail or fragment the
// device), and latency-critical loops that cannot afford the synchronisation an allocation
// implies.  This variant takes the same inputs and writes the same output, but keeps the
// candidate lists (and, for host output, the final candidates) in one file-scope device
// array of fixed size, so the call itself allocates nothing.
#include "ft_internal.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace {

// Fixed scratch shared by every call in the process, on every device that loads the
// library (the array lives until the process exits).
__device__ __align__(256) unsigned char g_noalloc_scratch[FT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once per device;
// in host code the array's name is only a host-side stand-in, never a device address).
int scratch_address(int device, void **out)
{
    if (device < 0 || device >= kMaxDevices)
        FT_FAIL(FT_ERR_RANGE, "topk_per_band_noalloc: device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_ptr[device] == nullptr) {
        void *p = nullptr;
        FT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return FT_OK;
}

}  // namespace

extern "C" int ft_topk_per_band_noalloc(ft_ctx *ctx, const ft_band *band, const ft_bank *bank,
                                        int k, ft_candidate *out, int out_on_device,
                                        void *stream)
{
    if (!ctx || !band || !bank || !out)
        FT_FAIL(FT_ERR_ARG, "topk_per_band_noalloc: null argument");
    if (band->ctx != ctx || bank->ctx != ctx || bank->band != band)
        FT_FAIL(FT_ERR_ARG, "topk_per_band_noalloc: band/bank do not belong together or to ctx");
    if (k < 1 || k > 32)
        FT_FAIL(FT_ERR_RANGE, "topk_per_band_noalloc: k must be in [1, 32]");
    int prev = -1;
    FT_CUDA(cudaGetDevice(&prev));
    if (prev != ctx->device)
        FT_CUDA(cudaSetDevice(ctx->device));
    (void)cudaGetLastError();  // drop errors left by earlier, unrelated runtime calls
    struct Restore {
        int dev;
        ~Restore()
        {
            if (dev >= 0)
                cudaSetDevice(dev);
        }
    } restore{prev != ctx->device ? prev : -1};
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const EvalShape sh = ft_default_shape(ctx, band, bank);
    const long long n_cta = ft_grid_ctas(bank, sh);
    const int lsub_max = std::min(bank->n_sub, (sh.J + bank->sub - 1) / bank->sub + 1);
    const size_t cand_bytes = static_cast<size_t>(n_cta) * lsub_max * k * sizeof(ft_candidate);
    const size_t out_bytes = static_cast<size_t>(bank->n_sub) * k * sizeof(ft_candidate);
    const size_t cand_off = 0;
    const size_t out_off = (cand_bytes + 255) / 256 * 256;
    const size_t need = out_on_device ? cand_bytes : out_off + out_bytes;
    if (need > FT_NOALLOC_SCRATCH_BYTES)
        FT_FAIL(FT_ERR_RANGE, "topk_per_band_noalloc: the search needs " + std::to_string(need) +
                                  " bytes of candidate scratch, above the fixed " +
                                  std::to_string(static_cast<size_t>(FT_NOALLOC_SCRATCH_BYTES)) +
                                  " bytes; use ft_topk_per_band or a smaller bank / k");

    void *base = nullptr;
    FT_TRY(scratch_address(ctx->device, &base));
    unsigned char *scr = static_cast<unsigned char *>(base);
    ft_candidate *dout = out_on_device ? out : reinterpret_cast<ft_candidate *>(scr + out_off);

    EvalParams p = ft_eval_base_params(band, bank);
    p.cand = reinterpret_cast<FtCand *>(scr + cand_off);
    p.k = k;
    p.sub = bank->sub;
    p.lsub_max = lsub_max;
    // every candidate slot the merge reads is written by the evaluation kernel first, so
    // the scratch needs no clearing between calls
    FT_TRY(ft_launch_eval(band, bank, sh, p, st));
    FT_TRY(ft_launch_merge(bank, sh, p.cand, k, lsub_max, dout, st));
    if (out_on_device)
        return FT_OK;
    FT_CUDA(cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, st));
    // synchronise, report and clear the device status word exactly as ft_topk_per_band does
    FT_TRY(ft_read_status(ctx, st));
    return FT_OK;
}
