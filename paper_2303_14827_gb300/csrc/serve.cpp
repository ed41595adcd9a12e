// serve.cpp -- serving entry points of libdqj (continuous batching).
#include "runtime.h"

using namespace dqj;

extern "C" {

dqj_status dqj_submit(dqj_ctx *ctx, const dqj_params *p, const dqj_outputs *out, dqj_ticket *ticket)
{
    (void)ctx; (void)p; (void)out; (void)ticket;
    return fail(DQJ_ERR_INVALID, "serving is not available in this build");
}

dqj_status dqj_poll(dqj_ctx *ctx, dqj_ticket ticket, int *done, dqj_status *result)
{
    (void)ctx; (void)ticket; (void)done; (void)result;
    return fail(DQJ_ERR_NOT_FOUND, "unknown ticket");
}

dqj_status dqj_destroy(dqj_ctx *ctx)
{
    if (!ctx) return fail(DQJ_ERR_INVALID, "ctx is NULL");
    cudaSetDevice(ctx->device);
    if (ctx->done_ev) cudaEventSynchronize(ctx->done_ev);
    if (ctx->host_stream) cudaStreamSynchronize(ctx->host_stream);
    scratch_free(ctx->scratch);
    if (ctx->host_planes) cudaFree(ctx->host_planes);
    if (ctx->host_stream) cudaStreamDestroy(ctx->host_stream);
    if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
    for (auto &v : ctx->ev)
        if (v) cudaEventDestroy(v);
    ctx->ev.clear();
    delete ctx;
    return DQJ_OK;
}

}  // extern "C"
