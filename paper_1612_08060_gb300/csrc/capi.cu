// capi.cu -- extern "C" entry points declared in include/napspmv.h.
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace nap {
int plan_create(const napspmv_csr *A, int32_t np, int32_t ppn, uint32_t flags, napspmv_plan_t **out);
}

using namespace nap;

static int arg_error(const char *msg)
{
    set_error(NAPSPMV_ERR_ARG, msg);
    return NAPSPMV_ERR_ARG;
}

extern "C" {

const char *napspmv_strerror(int code)
{
    switch (code) {
    case NAPSPMV_OK: return "ok";
    case NAPSPMV_ERR_ARG: return "invalid argument";
    case NAPSPMV_ERR_OOM: return "out of memory";
    case NAPSPMV_ERR_CUDA: return "CUDA error";
    case NAPSPMV_ERR_TIMEOUT: return "device-side wait timed out";
    case NAPSPMV_ERR_STATE: return "invalid state";
    case NAPSPMV_ERR_UNSUPPORTED: return "unsupported size";
    default: return "unknown error";
    }
}

int napspmv_plan(const napspmv_csr *A, int32_t n_p, int32_t ppn, uint32_t flags,
                 napspmv_plan_t **out)
{
    return plan_create(A, n_p, ppn, flags, out);
}

void napspmv_plan_destroy(napspmv_plan_t *P) { plan_free(P); }

int napspmv_apply_ex(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w,
                     int32_t reps, double scale, const napspmv_opts *opts, void *stream)
{
    if (!P) return arg_error("NULL plan");
    napspmv_ws_t *wl[1] = {ws};
    return apply_batch(1, &P, ws ? wl : nullptr, &v, &w, &reps, &scale, opts,
                       (cudaStream_t)stream);
}

int napspmv_apply(napspmv_plan_t *P, const double *v, double *w, void *stream)
{
    return napspmv_apply_ex(P, nullptr, v, w, 1, 1.0, nullptr, stream);
}

int napspmv_apply_n(napspmv_plan_t *P, const double *v, double *w, int32_t reps, double scale,
                    void *stream)
{
    return napspmv_apply_ex(P, nullptr, v, w, reps, scale, nullptr, stream);
}

int napspmv_apply_batch(int32_t count, napspmv_plan_t *const *plans, napspmv_ws_t *const *ws,
                        const double *const *v, double *const *w, const int32_t *reps,
                        const double *scale, const napspmv_opts *opts, void *stream)
{
    return apply_batch(count, plans, ws, v, w, reps, scale, opts, (cudaStream_t)stream);
}

int napspmv_ws_status(napspmv_ws_t *ws, void *stream)
{
    if (!ws) return arg_error("NULL workspace");
    NAP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    NAP_CUDA(cudaMemcpy(&h, ws->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        NAP_CUDA(cudaMemset(ws->err, 0, sizeof(int)));
        set_error(NAPSPMV_ERR_TIMEOUT, "a dependency wait of the fused kernel exceeded timeout_ms");
        return NAPSPMV_ERR_TIMEOUT;
    }
    return NAPSPMV_OK;
}

int napspmv_status(napspmv_plan_t *P, void *stream)
{
    if (!P) return arg_error("NULL plan");
    return napspmv_ws_status(P->ws, stream);
}

int napspmv_apply_host(napspmv_plan_t *P, const double *v_host, double *w_host, int32_t reps,
                       double scale, void *stream)
{
    if (!P || !v_host || !w_host) return arg_error("NULL plan or vector");
    cudaStream_t s = (cudaStream_t)stream;
    napspmv_ws_t *ws = P->ws;
    if (!ws->hv) {
        NAP_CUDA(cudaMalloc(&ws->hv, sizeof(double) * P->n));
        NAP_CUDA(cudaMalloc(&ws->hw, sizeof(double) * P->n));
    }
    NAP_CUDA(cudaMemcpyAsync(ws->hv, v_host, sizeof(double) * P->n, cudaMemcpyHostToDevice, s));
    int rc = napspmv_apply_ex(P, nullptr, ws->hv, ws->hw, reps, scale, nullptr, stream);
    if (rc) return rc;
    NAP_CUDA(cudaMemcpyAsync(w_host, ws->hw, sizeof(double) * P->n, cudaMemcpyDeviceToHost, s));
    return napspmv_ws_status(ws, stream);
}

int napspmv_ws_create(napspmv_plan_t *P, napspmv_ws_t **out)
{
    if (!P || !out) return arg_error("NULL plan or out");
    napspmv_ws_t *ws = new (std::nothrow) napspmv_ws_t();
    if (!ws) {
        set_error(NAPSPMV_ERR_OOM, "host allocation failed");
        return NAPSPMV_ERR_OOM;
    }
    int cur = 0;
    NAP_CUDA(cudaGetDevice(&cur));
    if (cur != P->device) NAP_CUDA(cudaSetDevice(P->device));
    int rc = ws_alloc(P, ws);
    if (cur != P->device) cudaSetDevice(cur);
    if (rc) {
        delete ws;
        return rc;
    }
    *out = ws;
    return NAPSPMV_OK;
}

void napspmv_ws_destroy(napspmv_ws_t *ws)
{
    if (!ws || ws->owned_by_plan) return;
    auto &G = ws->plan->graphs;  // graphs that captured this workspace's buffers
    for (size_t i = 0; i < G.size();) {
        if (G[i].ws == ws) {
            cudaGraphExecDestroy(G[i].exec);
            G.erase(G.begin() + i);
        } else {
            i++;
        }
    }
    ws_free(ws);
    delete ws;
}

int napspmv_plan_stats(const napspmv_plan_t *P, napspmv_stats *out)
{
    if (!P || !out) return arg_error("NULL plan or out");
    *out = P->stats;
    return NAPSPMV_OK;
}

int napspmv_plan_export(const napspmv_plan_t *P, int32_t which, int64_t *buf, int64_t *count)
{
    if (!P || !count) return arg_error("NULL plan or count");
    int64_t need = 0;
    if (which >= NAPSPMV_LIST_STD && which <= NAPSPMV_LIST_LBUF) {
        const HostList &L = P->lists[which];
        need = 2 + 2 * L.m + (L.m + 1) + L.total;
    } else if (which == NAPSPMV_LIST_TU) {
        need = 1 + 2 * (int64_t)P->send_proc.size();
    } else if (which == NAPSPMV_LIST_SPLIT) {
        need = 1 + 3 * P->n;
    } else {
        return arg_error("unknown list");
    }
    if (!buf) {
        *count = need;
        return NAPSPMV_OK;
    }
    if (*count < need) return arg_error("buffer too small");
    *count = need;
    if (which <= NAPSPMV_LIST_LBUF) {
        const HostList &L = P->lists[which];
        int64_t *o = buf;
        *o++ = L.m;
        *o++ = L.total;
        for (int64_t k = 0; k < L.m; k++) *o++ = L.src[k];
        for (int64_t k = 0; k < L.m; k++) *o++ = L.dst[k];
        for (int64_t k = 0; k <= L.m; k++) *o++ = L.ptr.empty() ? 0 : L.ptr[k];
        if (L.total) {
            std::vector<int32_t> h(L.total);
            NAP_CUDA(cudaMemcpy(h.data(), L.d_idx, sizeof(int32_t) * L.total, cudaMemcpyDeviceToHost));
            for (int64_t k = 0; k < L.total; k++) *o++ = h[k];
        }
    } else if (which == NAPSPMV_LIST_TU) {
        int64_t m = (int64_t)P->send_proc.size();
        buf[0] = m;
        for (int64_t k = 0; k < m; k++) {
            buf[1 + k] = P->send_proc[k];
            buf[1 + m + k] = P->recv_proc[k];
        }
    } else {
        std::vector<int32_t> h(3 * P->n);
        NAP_CUDA(cudaMemcpy(h.data(), P->d_split, sizeof(int32_t) * 3 * P->n, cudaMemcpyDeviceToHost));
        buf[0] = P->n;
        for (int64_t k = 0; k < 3 * P->n; k++) buf[1 + k] = h[k];
    }
    return NAPSPMV_OK;
}

int napspmv_get_default_opts(const napspmv_plan_t *P, napspmv_opts *out)
{
    if (!P || !out) return arg_error("NULL plan or out");
    *out = P->defaults;
    return NAPSPMV_OK;
}

int napspmv_set_default_opts(napspmv_plan_t *P, const napspmv_opts *opts)
{
    if (!P || !opts) return arg_error("NULL plan or opts");
    napspmv_opts o = resolve_opts(P, opts);
    o.debug_stall = 0;
    // every field is checked before it becomes a default (a bad timeout or
    // stage count would otherwise reach the kernels of later applies)
    if (int rc = check_opts(P, o)) return rc;
    int cur = 0;
    NAP_CUDA(cudaGetDevice(&cur));
    if (cur != P->device) NAP_CUDA(cudaSetDevice(P->device));
    int rc = build_items(P, o.tile_rows, o.tile_nnz);
    if (cur != P->device) cudaSetDevice(cur);
    if (rc) return rc;
    P->defaults = o;
    return NAPSPMV_OK;
}

}  // extern "C"
