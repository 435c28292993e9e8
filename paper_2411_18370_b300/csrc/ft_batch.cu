// ft_batch.cu -- many bands in one persistent launch, captured in a CUDA graph, with an
// autotuner for the launch shape.
//
// The work list is band-major: the tiles (sky point x f1 group x f0 tile) of band 0, then
// band 1, ... so that consecutive tickets hit the same band's power rows while they are
// hot in L2.  One persistent kernel takes tickets from a global counter; each CTA keeps
// running per-sub-band candidate lists for the band it works on and writes them out when
// it changes band.  A merge kernel reduces the per-CTA lists of every sub-band.  The
// sequence (reset counter, clear candidate slots, persistent kernel, merge) is captured
// once into a CUDA graph and replayed by ft_batch_run.
#include "ft_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

struct ft_batch {
    ft_ctx *ctx = nullptr;
    int device = 0;
    int n_bands = 0, k = 0, dtype = FT_F32;
    bool weighted = false;
    int F = 1, J = 32, nst = 2;
    std::vector<int> n_sub, S;
    std::vector<long long> tiles, sub_prefix_h;
    long long evals = 0;
    int n_sub_total = 0, n_sub_max = 0, lsub_max = 0;
    EvalParams *d_params = nullptr;
    long long *d_prefix = nullptr;
    int *d_nsub = nullptr, *d_subprefix = nullptr;
    unsigned long long *d_counter = nullptr;
    ft_candidate *d_scr = nullptr, *d_out = nullptr;
    size_t scr_bytes = 0, smem = 0;
    int grid = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != d)
            cudaSetDevice(d);
        (void)cudaGetLastError();
    }
    ~DevGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

void free_batch(ft_batch *b)
{
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    if (b->cap)
        cudaStreamDestroy(b->cap);
    cudaFree(b->d_params);
    cudaFree(b->d_prefix);
    cudaFree(b->d_nsub);
    cudaFree(b->d_subprefix);
    cudaFree(b->d_counter);
    cudaFree(b->d_scr);
    cudaFree(b->d_out);
    delete b;
}

int check_inputs(ft_ctx *ctx, int n, const ft_band *const *bands, const ft_bank *const *banks, int k)
{
    if (!ctx || n < 1 || !bands || !banks)
        FT_FAIL(FT_ERR_ARG, "batch: null argument or no bands");
    if (k < 1 || k > 32)
        FT_FAIL(FT_ERR_RANGE, "batch: k must be in [1, 32]");
    for (int i = 0; i < n; ++i) {
        if (!bands[i] || !banks[i] || bands[i]->ctx != ctx || banks[i]->ctx != ctx ||
            banks[i]->band != bands[i])
            FT_FAIL(FT_ERR_ARG, "batch: band/bank " + std::to_string(i) + " invalid or mismatched");
        if (bands[i]->dtype != bands[0]->dtype ||
            ft_band_weighted(bands[i]) != ft_band_weighted(bands[0]) ||
            (bands[i]->d_D && !banks[i]->d_sky_inv))
            FT_FAIL(FT_ERR_ARG, "batch: all bands must share storage type and weighting");
        if (!banks[i]->window_safe)
            FT_FAIL(FT_ERR_ARG, "batch: bank " + std::to_string(i) +
                                    " has tracks that may leave its window (widen the wings)");
    }
    return FT_OK;
}

// Rows per stage: the largest multiple of 4 (<= 32) whose nst stages of Ws-bin windows fit
// 80 KB.
int rows_for(int Ws, int nst)
{
    const int rb = Ws * 4;
    int S = (80 * 1024) / (nst * rb);
    S = std::min(S, 32);
    S &= ~3;
    return std::max(S, 4);
}

// Build the work tables and the graph.  cap_frac < 1 keeps only that fraction of each
// band's tiles (at least one), for timing candidate shapes.
int build(ft_ctx *ctx, int n, const ft_band *const *bands, const ft_bank *const *banks, int k,
          int J, int nst, double cap_frac, ft_batch **out)
{
    ft_batch *b = new ft_batch;
    b->ctx = ctx;
    b->device = ctx->device;
    b->n_bands = n;
    b->k = k;
    b->dtype = bands[0]->dtype;
    b->weighted = ft_band_weighted(bands[0]);
    b->J = J;
    b->nst = nst;
    // per band: P sky points x F1 f1 values per CTA; the CTA has the most warps any band
    // uses (a band with fewer leaves the rest idle)
    std::vector<int> bP(n), bF1(n);
    int F = 1;
    for (int i = 0; i < n; ++i) {
        ft_sky_grouping(banks[i], 20, &bP[i], &bF1[i]);
        F = std::max(F, bP[i] * bF1[i]);
    }
    b->F = F;
    const bool pair = b->dtype != FT_F32;
    if (J % (pair ? 64 : 32) != 0 || J < 32 || J > 256 || nst < 2 || nst > 4) {
        free_batch(b);
        FT_FAIL(FT_ERR_RANGE, "batch: unsupported tile width / stages");
    }
    std::vector<EvalParams> params(n);
    std::vector<long long> prefix(n + 1, 0);
    std::vector<int> sub_prefix(n + 1, 0);
    size_t tile_smem = 0;
    for (int i = 0; i < n; ++i) {
        const ft_band *bd = bands[i];
        const ft_bank *bk = banks[i];
        EvalParams &p = params[i];
        p = ft_eval_base_params(bd, bk);
        p.status = ctx->d_status;
        p.P = bP[i];
        p.F1 = bF1[i];
        p.n_skyg = (bk->n_sky + bP[i] - 1) / bP[i];
        p.sky_order = bP[i] > 1 ? bk->d_sky_order : nullptr;
        p.k = k;
        p.sub = bk->sub;
        const int Ws = ft_window_bins(bd, bk, J, bP[i]);
        const int S = rows_for(Ws, nst);
        b->S.push_back(S);
        p.S = S;
        p.nst = nst;
        p.row_bytes = ft_batch_row_bytes(bd);
        p.Wp = bd->Wp;
        p.Ws = Ws;
        p.srow_bytes = Ws * 4;
        ft_encode_rows_map(bd, Ws, S, &p.rows_map, &p.rows_map_ok);  // (never fails: ok = 0 instead)
        p.row_elems = bd->dtype == FT_F32 ? bd->Wp : 2 * bd->Wp;
        p.n_stages = static_cast<int>((bd->N + S - 1) / S);
        p.n_f0t = (bk->n_f0 + J - 1) / J;
        p.n_f1g = (bk->n_f1 + bF1[i] - 1) / bF1[i];
        p.lsub_max = std::min(bk->n_sub, (J + bk->sub - 1) / bk->sub + 1);
        const long long T = p.n_skyg * p.n_f1g * static_cast<long long>(p.n_f0t);
        long long Tc = T;
        if (cap_frac < 1.0)
            Tc = std::max<long long>(1, static_cast<long long>(std::ceil(T * cap_frac)));
        b->tiles.push_back(Tc);
        prefix[i + 1] = prefix[i] + Tc;
        const long long nt = bk->n_sky * bk->n_f1 * static_cast<long long>(bk->n_f0);
        b->evals += static_cast<long long>(static_cast<double>(nt) * Tc / T) * bd->N;
        b->n_sub.push_back(bk->n_sub);
        sub_prefix[i + 1] = sub_prefix[i] + bk->n_sub;
        b->n_sub_max = std::max(b->n_sub_max, bk->n_sub);
        b->lsub_max = std::max(b->lsub_max, p.lsub_max);
        tile_smem = std::max(tile_smem, ft_batch_tile_smem(Ws, S, F, bP[i], J, nst, ft_band_weighted(bands[0])));
    }
    b->n_sub_total = sub_prefix[n];
    b->sub_prefix_h.assign(sub_prefix.begin(), sub_prefix.end());
    const size_t list_off = (tile_smem + 15) / 16 * 16;
    b->smem = list_off + static_cast<size_t>(b->lsub_max + b->n_sub_max) * k * sizeof(ft_candidate);
    if (b->smem > ctx->smem_optin) {
        free_batch(b);
        FT_FAIL(FT_ERR_RANGE, "batch: shared memory for this shape exceeds the device limit");
    }
    BatchParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.n_bands = n;
    bp.k = k;
    bp.n_sub_max = b->n_sub_max;
    bp.lsub_max = b->lsub_max;
    bp.list_off = list_off;
    int rc = ft_launch_batched(b->dtype, b->weighted, J, F, bp, b->smem, &b->grid, false, nullptr);
    if (rc != FT_OK) {
        free_batch(b);
        return rc;
    }
    b->scr_bytes = static_cast<size_t>(b->grid) * n * b->n_sub_max * k * sizeof(ft_candidate);
    auto fail = [&](cudaError_t e, const char *what) {
        ft_set_error(std::string("batch: ") + what + ": " + cudaGetErrorString(e));
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? FT_ERR_OOM : FT_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_params, n * sizeof(EvalParams))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_prefix, (n + 1) * sizeof(long long))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_nsub, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_subprefix, (n + 1) * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_counter, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_scr, b->scr_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_out, static_cast<size_t>(b->n_sub_total) * k * sizeof(ft_candidate))) !=
            cudaSuccess)
        return fail(e, "allocation");
    for (int i = 0; i < n; ++i)
        params[i].cand = reinterpret_cast<FtCand *>(b->d_scr);  // non-null: selection on
    if ((e = cudaMemcpy(b->d_params, params.data(), n * sizeof(EvalParams), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(b->d_prefix, prefix.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(b->d_nsub, b->n_sub.data(), n * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_subprefix, sub_prefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return fail(e, "upload");
    bp.params = b->d_params;
    bp.tile_prefix = b->d_prefix;
    bp.n_sub = b->d_nsub;
    bp.counter = b->d_counter;
    bp.scr = b->d_scr;
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(e, "stream");
    if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return fail(e, "begin capture");
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), b->cap);
    cudaMemsetAsync(b->d_scr, 0xff, b->scr_bytes, b->cap);  // every slot empty (index -1)
    int g2 = 0;
    const int rc1 = ft_launch_batched(b->dtype, b->weighted, J, F, bp, b->smem, &g2, true, b->cap);
    const int rc2 = ft_launch_merge_persist(b->d_scr, b->grid, n, b->n_sub_max, k, b->d_subprefix,
                                            b->n_sub_total, b->d_out, b->cap);
    const cudaError_t ec = cudaStreamEndCapture(b->cap, &b->graph);
    if (rc1 != FT_OK || rc2 != FT_OK) {
        free_batch(b);
        return rc1 != FT_OK ? rc1 : rc2;
    }
    if (ec != cudaSuccess)
        return fail(ec, "end capture");
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess)
        return fail(e, "graph instantiate");
    *out = b;
    return FT_OK;
}

int time_run(ft_batch *b, float *ms)
{
    cudaEvent_t e0, e1;
    FT_CUDA(cudaEventCreate(&e0));
    FT_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        FT_CUDA(cudaEventRecord(e0, b->cap));
        FT_CUDA(cudaGraphLaunch(b->exec, b->cap));
        FT_CUDA(cudaEventRecord(e1, b->cap));
        FT_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        FT_CUDA(cudaEventElapsedTime(&t, e0, e1));
        if (rep > 0)
            best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return FT_OK;
}

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;  // key -> (J, nst)

std::string tune_key(int n, const ft_band *const *bands, const ft_bank *const *banks, int k)
{
    // storage type, weighting, rows, the set of window widths (rounded) and f1 counts
    std::string key = std::to_string(bands[0]->dtype) + (ft_band_weighted(bands[0]) ? "w" : "u") + "k" +
                      std::to_string(k);
    std::vector<int> wb;
    long long nrows = 0;
    int nf1 = 0;
    for (int i = 0; i < n; ++i) {
        wb.push_back((bands[i]->W + 63) / 64);
        nrows = std::max<long long>(nrows, bands[i]->N);
        nf1 = std::max(nf1, banks[i]->n_f1);
    }
    std::sort(wb.begin(), wb.end());
    wb.erase(std::unique(wb.begin(), wb.end()), wb.end());
    key += "n" + std::to_string(nrows / 1024) + "f" + std::to_string(nf1) + "W";
    for (int w : wb)
        key += std::to_string(w) + ",";
    return key;
}

// Time each candidate (tile width, stages) on a capped subset of every band's tiles; the
// subset has the same composition as the full list, so the fastest candidate per
// evaluation wins.
int autotune(ft_ctx *ctx, int n, const ft_band *const *bands, const ft_bank *const *banks, int k,
             int *J_out, int *nst_out)
{
    const std::string key = tune_key(n, bands, banks, k);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *J_out = it->second.first;
            *nst_out = it->second.second;
            return FT_OK;
        }
    }
    long long total = 0;
    for (int i = 0; i < n; ++i)
        total += banks[i]->n_sky;  // order of magnitude of tiles
    const double frac = std::min(1.0, std::max(0.01, 6000.0 / std::max<long long>(total, 1)));
    const int Js[] = {128, 192, 256};
    const int nsts[] = {2, 3};
    double best_rate = -1.0;
    int bJ = 256, bN = 2;
    for (int J : Js) {
        for (int nst : nsts) {
            ft_batch *b = nullptr;
            if (build(ctx, n, bands, banks, k, J, nst, frac, &b) != FT_OK)
                continue;  // shape does not fit: skip it
            float ms = 0.f;
            const int rc = time_run(b, &ms);
            const double rate = rc == FT_OK && ms > 0 ? b->evals / (ms * 1e-3) : -1.0;
            free_batch(b);
            if (rc != FT_OK)
                return rc;
            if (rate > best_rate) {
                best_rate = rate;
                bJ = J;
                bN = nst;
            }
        }
    }
    if (best_rate < 0)
        FT_FAIL(FT_ERR_RANGE, "batch: no candidate launch shape fits these bands");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {bJ, bN};
    *J_out = bJ;
    *nst_out = bN;
    return FT_OK;
}

}  // namespace

extern "C" {

int ft_batch_create(ft_ctx *ctx, int n_bands, const ft_band *const *bands,
                    const ft_bank *const *banks, int k, const ft_tune *tune, void *stream,
                    ft_batch **out)
{
    if (!out)
        FT_FAIL(FT_ERR_ARG, "batch: null out");
    *out = nullptr;
    FT_TRY(check_inputs(ctx, n_bands, bands, banks, k));
    DevGuard g(ctx->device);
    if (stream)
        FT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int J = 0, nst = 0;
    if (tune && tune->tile_f0 > 0)
        J = tune->tile_f0;
    if (tune && tune->stages > 0)
        nst = tune->stages;
    if (J == 0 || nst == 0) {
        int aJ = 256, aN = 2;
        FT_TRY(autotune(ctx, n_bands, bands, banks, k, &aJ, &aN));
        J = J ? J : aJ;
        nst = nst ? nst : aN;
    }
    return build(ctx, n_bands, bands, banks, k, J, nst, 1.0, out);
}

int ft_batch_run(ft_batch *b, ft_candidate *out, int out_on_device, void *stream)
{
    if (!b || !out)
        FT_FAIL(FT_ERR_ARG, "batch_run: null argument");
    DevGuard g(b->ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FT_CUDA(cudaGraphLaunch(b->exec, st));
    const size_t bytes = static_cast<size_t>(b->n_sub_total) * b->k * sizeof(ft_candidate);
    FT_CUDA(cudaMemcpyAsync(out, b->d_out, bytes,
                            out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (out_on_device)
        return FT_OK;
    return ft_check_status(b->ctx, stream);
}

int ft_batch_info(const ft_batch *b, int64_t *n_candidates, int64_t *evals, ft_tune *chosen,
                  int *n_ctas)
{
    if (!b)
        FT_FAIL(FT_ERR_ARG, "batch_info: null batch");
    if (n_candidates)
        *n_candidates = static_cast<int64_t>(b->n_sub_total) * b->k;
    if (evals)
        *evals = b->evals;
    if (chosen) {
        chosen->tile_f0 = b->J;
        chosen->stages = b->nst;
        chosen->rows_per_stage = b->S.empty() ? 0 : *std::max_element(b->S.begin(), b->S.end());
    }
    if (n_ctas)
        *n_ctas = b->grid;
    return FT_OK;
}

void ft_batch_destroy(ft_batch *b)
{
    if (!b)
        return;
    DevGuard g(b->device);
    free_batch(b);
}

int ft_eval_batched(ft_ctx *ctx, int n_bands, const ft_band *const *bands,
                    const ft_bank *const *banks, int k, ft_candidate *out, int out_on_device,
                    const ft_tune *tune, void *stream)
{
    ft_batch *b = nullptr;
    FT_TRY(ft_batch_create(ctx, n_bands, bands, banks, k, tune, stream, &b));
    const int rc = ft_batch_run(b, out, out_on_device, stream);
    if (out_on_device && stream)
        cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    else if (out_on_device)
        cudaDeviceSynchronize();
    ft_batch_destroy(b);
    return rc;
}

}  // extern "C"
