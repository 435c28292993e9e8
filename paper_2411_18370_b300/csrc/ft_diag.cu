// ft_diag.cu -- failure-detection self-test: a bounded wait that runs out on purpose.
//
// One CTA waits on an mbarrier whose only expected arrival never comes.  The wait gives up
// after about one second of %globaltimer, the kernel records FT_STATUS_TIMEOUT like a search
// kernel whose copies never landed, and returns; nothing faults or hangs.

#include "ft_internal.cuh"
#include "ft_ptx.cuh"

namespace {

__global__ void k_wait_never(unsigned *status, unsigned long long *ns_out)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        ftp::mbar_init(&bar, 1);
        ftp::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = ftp::global_ns();
        const bool ok = ftp::mbar_wait_bounded(&bar, 0);
        *ns_out = ftp::global_ns() - t0;
        if (!ok)
            atomicOr(status, FT_STATUS_TIMEOUT);
    }
}

}  // namespace

int ft_selftest_bounded_wait(ft_ctx *ctx, double *waited_s, void *stream)
{
    if (!ctx)
        FT_FAIL(FT_ERR_ARG, "selftest_bounded_wait: null ctx");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess)
        prev = -1;
    if (prev != ctx->device)
        FT_CUDA(cudaSetDevice(ctx->device));
    (void)cudaGetLastError();
    struct Restore {
        int d;
        ~Restore()
        {
            if (d >= 0)
                cudaSetDevice(d);
        }
    } restore{prev != ctx->device ? prev : -1};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *buf = nullptr;
    FT_TRY(ft_ctx_outbuf(ctx, sizeof(unsigned long long), &buf));
    unsigned long long *d_ns = static_cast<unsigned long long *>(buf);
    k_wait_never<<<1, 32, 0, st>>>(ctx->d_status, d_ns);
    FT_CUDA(cudaGetLastError());
    unsigned long long ns = 0;
    FT_CUDA(cudaMemcpyAsync(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost, st));
    FT_CUDA(cudaStreamSynchronize(st));
    if (waited_s)
        *waited_s = static_cast<double>(ns) * 1e-9;
    return ft_read_status(ctx, st);
}
