// bri_apply_host: the stencil apply on spinors that live in host memory.
//
// The input is copied to the device in slabs of whole time slices on one
// stream; each slab of the output is computed as soon as the slab and its two
// neighbours in t (the stencil reaches one time slice in each direction) have
// arrived, and copied back on a third stream.  Host-to-device copies, the
// stencil and device-to-host copies of different slabs overlap.  The last
// slab in t needs slab 0 and slab 0 needs the last one, so the compute order is
// 1, 2, ..., K-1, 0.  Device staging buffers belong to the context.
#include <vector>

#include "ctx.h"

bri_status bri_dslash_range(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode, bri_prec prec,
                            int s0, int s1, cudaStream_t s);

struct HostApplyWork {
    void *din = nullptr, *dout = nullptr;
    size_t cap = 0;
    cudaStream_t h2d = nullptr, comp[2] = {nullptr, nullptr}, d2h = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_out;
    cudaEvent_t start = nullptr, done = nullptr;
};

void bri_host_apply_free(bri_ctx *ctx) {
    HostApplyWork *w = ctx->hw;
    if (!w) return;
    for (cudaStream_t s : {w->h2d, w->comp[0], w->comp[1], w->d2h})
        if (s) cudaStreamSynchronize(s);
    if (w->din) cudaFree(w->din);
    if (w->dout) cudaFree(w->dout);
    for (auto e : w->ev_in) cudaEventDestroy(e);
    for (auto e : w->ev_out) cudaEventDestroy(e);
    if (w->start) cudaEventDestroy(w->start);
    if (w->done) cudaEventDestroy(w->done);
    for (cudaStream_t s : {w->h2d, w->comp[0], w->comp[1], w->d2h})
        if (s) cudaStreamDestroy(s);
    delete w;
    ctx->hw = nullptr;
}

static constexpr int MAX_SLABS = 32;

static bri_status ensure_host_work(bri_ctx *ctx, size_t bytes) {
    HostApplyWork *w = ctx->hw;
    if (!w) {
        w = new HostApplyWork();
        ctx->hw = w;
        for (cudaStream_t *s : {&w->h2d, &w->comp[0], &w->comp[1], &w->d2h})
            BRI_TRY_CUDA(ctx, cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
        w->ev_in.resize(MAX_SLABS);
        w->ev_out.resize(MAX_SLABS);
        for (auto &e : w->ev_in) BRI_TRY_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : w->ev_out) BRI_TRY_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        BRI_TRY_CUDA(ctx, cudaEventCreateWithFlags(&w->start, cudaEventDisableTiming));
        BRI_TRY_CUDA(ctx, cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming));
    }
    if (w->cap < bytes) {
        // earlier calls may still be reading or writing the staging buffers
        for (cudaStream_t s : {w->h2d, w->comp[0], w->comp[1], w->d2h}) BRI_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        if (w->din) cudaFree(w->din);
        if (w->dout) cudaFree(w->dout);
        w->din = w->dout = nullptr;
        w->cap = 0;
        BRI_TRY_CUDA(ctx, cudaMalloc(&w->din, bytes));
        BRI_TRY_CUDA(ctx, cudaMalloc(&w->dout, bytes));
        w->cap = bytes;
    }
    return BRI_OK;
}

bri_status bri_apply_host_impl(bri_ctx *ctx, void *out, const void *in, int nrhs, double m0, int mode,
                               bri_prec prec, cudaStream_t user) {
    const bri::Geom &g = ctx->g;
    const size_t elt = prec == BRI_F64 ? 16 : 8;
    const size_t per_rhs = elt * 12 * (size_t)g.V;
    BRI_RETURN_IF(ensure_host_work(ctx, per_rhs * nrhs));
    HostApplyWork *w = ctx->hw;
    const int Lt = g.L[3];
    const int K = Lt < MAX_SLABS ? Lt : MAX_SLABS;
    const size_t S3 = (size_t)g.L[0] * g.L[1] * g.L[2];
    int tb[MAX_SLABS + 1];
    for (int k = 0; k <= K; k++) tb[k] = (int)((long)k * Lt / K);
    // work enqueued on the caller's stream before this call comes first
    BRI_TRY_CUDA(ctx, cudaEventRecord(w->start, user));
    for (cudaStream_t s : {w->h2d, w->comp[0], w->comp[1], w->d2h})
        BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(s, w->start, 0));
    for (int r = 0; r < nrhs; r++) {
        char *din = (char *)w->din + r * per_rhs, *dout = (char *)w->dout + r * per_rhs;
        const char *hin = (const char *)in + r * per_rhs;
        char *hout = (char *)out + r * per_rhs;
        for (int k = 0; k < K; k++) {
            const size_t o = (size_t)tb[k] * S3 * 12 * elt, n = (size_t)(tb[k + 1] - tb[k]) * S3 * 12 * elt;
            BRI_TRY_CUDA(ctx, cudaMemcpyAsync(din + o, hin + o, n, cudaMemcpyHostToDevice, w->h2d));
            BRI_TRY_CUDA(ctx, cudaEventRecord(w->ev_in[k], w->h2d));
        }
        for (int i = 1; i <= K; i++) {
            const int k = i % K;
            // slabs alternate between two compute streams so that the tail of one
            // slab's grid overlaps the start of the next
            cudaStream_t cs = w->comp[i & 1];
            const int need[3] = {(k + K - 1) % K, k, (k + 1) % K};
            for (int nb : need) BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(cs, w->ev_in[nb], 0));
            BRI_RETURN_IF(bri_dslash_range(ctx, dout, din, 1, m0, mode, prec, (int)(tb[k] * S3), (int)(tb[k + 1] * S3),
                                           cs));
            BRI_TRY_CUDA(ctx, cudaEventRecord(w->ev_out[k], cs));
            BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(w->d2h, w->ev_out[k], 0));
            const size_t o = (size_t)tb[k] * S3 * 12 * elt, n = (size_t)(tb[k + 1] - tb[k]) * S3 * 12 * elt;
            BRI_TRY_CUDA(ctx, cudaMemcpyAsync(hout + o, dout + o, n, cudaMemcpyDeviceToHost, w->d2h));
        }
    }
    // the next call's input copies must not overwrite slabs still being read
    BRI_TRY_CUDA(ctx, cudaEventRecord(w->done, w->d2h));
    BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(w->h2d, w->done, 0));
    BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(w->comp[0], w->done, 0));
    BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(w->comp[1], w->done, 0));
    BRI_TRY_CUDA(ctx, cudaStreamWaitEvent(user, w->done, 0));
    return BRI_OK;
}
