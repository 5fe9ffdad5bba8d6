// solve.cu -- deterministic FP64 dot products, CG and CG with iterative
// refinement on top of the node-aware apply.
//
// Precision scheme: the matrix used inside the inner CG is the FP32 copy of
// A's values (FP32 products, FP64 sums); every vector, dot product and the
// outer residual r = b - A x stay FP64, the outer residual using the FP64
// values.  Each dot product sums over a fixed partition in a fixed order, so
// its value does not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace nap {
namespace {

constexpr int kDotBlocks = 1024;  // fixed grid: the partition of every dot product
constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (kThreads / 32) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;  // valid in thread 0
}

// Partial sums per block over indices i = b*256 + t + q*1024*256; the last
// block to finish adds the 1024 partials in index order and resets the ticket.
__global__ void __launch_bounds__(kThreads)
    k_dot(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
          double *partial, unsigned *ticket, double *result)
{
    __shared__ double sh[kThreads / 32];
    __shared__ bool last;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)kDotBlocks * kThreads)
        s = fma(x[i], y[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == kDotBlocks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0;
    for (int b = threadIdx.x; b < kDotBlocks; b += kThreads) a += __ldcg(partial + b);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) {
        *result = a;
        *ticket = 0;
    }
}

struct Scal {
    double rr, rr_new, pq, alpha, beta, bb, rnorm0;
};

__global__ void k_alpha(Scal *s) { s->alpha = s->rr / s->pq; }
__global__ void k_beta(Scal *s)
{
    s->beta = s->rr_new / s->rr;
    s->rr = s->rr_new;
}

// x += alpha p ; r -= alpha q
__global__ void k_update_xr(double *x, double *r, const double *p, const double *q, int64_t n,
                            const Scal *s)
{
    const double a = s->alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(a, p[i], x[i]);
        r[i] = fma(-a, q[i], r[i]);
    }
}
// p = r + beta p
__global__ void k_update_p(double *p, const double *r, int64_t n, const Scal *s)
{
    const double b = s->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(b, p[i], r[i]);
}
// r = b - q ; p = r
__global__ void k_resid(double *r, double *p, const double *b, const double *q, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[i] - q[i];
        r[i] = v;
        if (p) p[i] = v;
    }
}
// x += d
__global__ void k_add(double *x, const double *d, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

struct DotScratch {
    double *partial = nullptr;
    unsigned *ticket = nullptr;
};

int dot_launch(const double *x, const double *y, int64_t n, double *result, DotScratch &ds,
               cudaStream_t s)
{
    k_dot<<<kDotBlocks, kThreads, 0, s>>>(x, y, n, ds.partial, ds.ticket, result);
    count_launch(1);
    NAP_CUDA(cudaGetLastError());
    return NAPSPMV_OK;
}

struct CgBuffers {
    double *r = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
    Scal *sc = nullptr;
    DotScratch ds;
    cudaStream_t s = 0;
    ~CgBuffers()
    {
        void *ptrs[] = {r, p, q, d, sc, ds.partial, ds.ticket};
        for (void *x : ptrs)
            if (x) cudaFreeAsync(x, s);
    }
};

int cg_alloc(CgBuffers &B, int64_t n, cudaStream_t s)
{
    B.s = s;
    NAP_CUDA(cudaMallocAsync(&B.r, sizeof(double) * n, s));
    NAP_CUDA(cudaMallocAsync(&B.p, sizeof(double) * n, s));
    NAP_CUDA(cudaMallocAsync(&B.q, sizeof(double) * n, s));
    NAP_CUDA(cudaMallocAsync(&B.d, sizeof(double) * n, s));
    NAP_CUDA(cudaMallocAsync(&B.sc, sizeof(Scal), s));
    NAP_CUDA(cudaMallocAsync(&B.ds.partial, sizeof(double) * kDotBlocks, s));
    NAP_CUDA(cudaMallocAsync(&B.ds.ticket, sizeof(unsigned), s));
    NAP_CUDA(cudaMemsetAsync(B.ds.ticket, 0, sizeof(unsigned), s));
    NAP_CUDA(cudaMemsetAsync(B.sc, 0, sizeof(Scal), s));
    return NAPSPMV_OK;
}

int grid_for(const napspmv_plan_t *P, int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)P->num_sms * 8));
}

// CG on A x = b from the x given, with the apply options `o`.  Stops when the
// recursive residual satisfies ||r|| <= rtol * ||b|| or after max_it
// iterations (checked on the host every `poll` iterations).  x, b: device.
int cg_core(napspmv_plan_t *P, const double *b, double *x, double rtol, int max_it,
            const napspmv_opts &o, CgBuffers &B, int *iters)
{
    cudaStream_t s = B.s;
    const int64_t n = P->n;
    const int g = grid_for(P, n);
    int rc;
    if ((rc = napspmv_apply_ex(P, nullptr, x, B.q, 1, 1.0, &o, s))) return rc;
    k_resid<<<g, 256, 0, s>>>(B.r, B.p, b, B.q, n);
    count_launch(1);
    if ((rc = dot_launch(b, b, n, &B.sc->bb, B.ds, s))) return rc;
    if ((rc = dot_launch(B.r, B.r, n, &B.sc->rr, B.ds, s))) return rc;
    Scal h{};
    NAP_CUDA(cudaMemcpyAsync(&h, B.sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
    NAP_CUDA(cudaStreamSynchronize(s));
    const double bn = h.bb > 0 ? std::sqrt(h.bb) : 1.0;
    int it = 0;
    const int poll = 8;
    bool done = std::sqrt(h.rr) <= rtol * bn;
    while (!done && it < max_it) {
        for (int q = 0; q < poll && it < max_it; q++, it++) {
            if ((rc = napspmv_apply_ex(P, nullptr, B.p, B.q, 1, 1.0, &o, s))) return rc;
            if ((rc = dot_launch(B.p, B.q, n, &B.sc->pq, B.ds, s))) return rc;
            k_alpha<<<1, 1, 0, s>>>(B.sc);
            k_update_xr<<<g, 256, 0, s>>>(x, B.r, B.p, B.q, n, B.sc);
            count_launch(2);
            if ((rc = dot_launch(B.r, B.r, n, &B.sc->rr_new, B.ds, s))) return rc;
            k_beta<<<1, 1, 0, s>>>(B.sc);
            k_update_p<<<g, 256, 0, s>>>(B.p, B.r, n, B.sc);
            count_launch(2);
        }
        NAP_CUDA(cudaGetLastError());
        NAP_CUDA(cudaMemcpyAsync(&h, B.sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
        NAP_CUDA(cudaStreamSynchronize(s));
        if ((rc = napspmv_ws_status(P->ws, s))) return rc;
        if (!std::isfinite(h.rr)) break;
        done = std::sqrt(h.rr) <= rtol * bn;
    }
    *iters = it;
    return NAPSPMV_OK;
}

// ||b - A x|| / ||b|| in FP64 with the FP64 apply; leaves r = b - A x in B.r.
int true_relres(napspmv_plan_t *P, const double *b, const double *x, CgBuffers &B, double *out)
{
    cudaStream_t s = B.s;
    napspmv_opts o = P->defaults;
    o.precision = NAPSPMV_PREC_F64;
    int rc;
    if ((rc = napspmv_apply_ex(P, nullptr, x, B.q, 1, 1.0, &o, s))) return rc;
    k_resid<<<grid_for(P, P->n), 256, 0, s>>>(B.r, nullptr, b, B.q, P->n);
    count_launch(1);
    if ((rc = dot_launch(B.r, B.r, P->n, &B.sc->rnorm0, B.ds, s))) return rc;
    if ((rc = dot_launch(b, b, P->n, &B.sc->bb, B.ds, s))) return rc;
    Scal h{};
    NAP_CUDA(cudaMemcpyAsync(&h, B.sc, sizeof(Scal), cudaMemcpyDeviceToHost, s));
    NAP_CUDA(cudaStreamSynchronize(s));
    if ((rc = napspmv_ws_status(P->ws, s))) return rc;
    *out = std::sqrt(h.rnorm0) / (h.bb > 0 ? std::sqrt(h.bb) : 1.0);
    return NAPSPMV_OK;
}

}  // namespace
}  // namespace nap

using namespace nap;

extern "C" {

int napspmv_dot(const double *x, const double *y, int64_t n, double *result, void *stream)
{
    if ((n > 0 && (!x || !y)) || !result || n < 0) {
        set_error(NAPSPMV_ERR_ARG, "NULL vector or result, or n < 0");
        return NAPSPMV_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DotScratch ds;
    NAP_CUDA(cudaMallocAsync(&ds.partial, sizeof(double) * kDotBlocks, s));
    NAP_CUDA(cudaMallocAsync(&ds.ticket, sizeof(unsigned), s));
    NAP_CUDA(cudaMemsetAsync(ds.ticket, 0, sizeof(unsigned), s));
    int rc = dot_launch(x, y, n, result, ds, s);
    cudaFreeAsync(ds.partial, s);
    cudaFreeAsync(ds.ticket, s);
    return rc;
}

int napspmv_cg(napspmv_plan_t *P, const double *b, double *x, double rtol, int32_t max_it,
               napspmv_cg_info *info, void *stream)
{
    if (!P || !b || !x || max_it < 0 || !(rtol > 0)) {
        set_error(NAPSPMV_ERR_ARG, "NULL plan or vector, max_it < 0 or rtol <= 0");
        return NAPSPMV_ERR_ARG;
    }
    CgBuffers B;
    int rc = cg_alloc(B, P->n, (cudaStream_t)stream);
    if (rc) return rc;
    napspmv_opts o = P->defaults;
    o.precision = NAPSPMV_PREC_F64;
    int it = 0;
    if ((rc = cg_core(P, b, x, rtol, max_it, o, B, &it))) return rc;
    double rr = 0;
    if ((rc = true_relres(P, b, x, B, &rr))) return rc;
    if (info) {
        info->outer_iters = 1;
        info->inner_iters = it;
        info->relres = rr;
        info->converged = rr <= rtol;
    }
    return NAPSPMV_OK;
}

int napspmv_cg_ir(napspmv_plan_t *P, const double *b, double *x, double rtol, double inner_rtol,
                  int32_t max_outer, int32_t inner_max, napspmv_cg_info *info, void *stream)
{
    if (!P || !b || !x || max_outer < 1 || inner_max < 1 || !(rtol > 0) || !(inner_rtol > 0)) {
        set_error(NAPSPMV_ERR_ARG, "bad arguments to napspmv_cg_ir");
        return NAPSPMV_ERR_ARG;
    }
    if (!P->d_val32) {
        set_error(NAPSPMV_ERR_STATE, "plan was built without NAPSPMV_F32_VALUES");
        return NAPSPMV_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CgBuffers B, I;
    int rc = cg_alloc(B, P->n, s);
    if (rc) return rc;
    if ((rc = cg_alloc(I, P->n, s))) return rc;
    napspmv_opts o32 = P->defaults;
    o32.precision = NAPSPMV_PREC_F32;
    int outer = 0, inner_total = 0;
    double rr = 0;
    for (;;) {
        if ((rc = true_relres(P, b, x, B, &rr))) return rc;  // B.r = b - A x (FP64)
        if (rr <= rtol || outer >= max_outer || !std::isfinite(rr)) break;
        // inner solve A d = r with FP32-stored values, d_0 = 0
        NAP_CUDA(cudaMemsetAsync(I.d, 0, sizeof(double) * P->n, s));
        int it = 0;
        if ((rc = cg_core(P, B.r, I.d, inner_rtol, inner_max, o32, I, &it))) return rc;
        k_add<<<grid_for(P, P->n), 256, 0, s>>>(x, I.d, P->n);
        count_launch(1);
        NAP_CUDA(cudaGetLastError());
        inner_total += it;
        outer++;
    }
    if (info) {
        info->outer_iters = outer;
        info->inner_iters = inner_total;
        info->relres = rr;
        info->converged = rr <= rtol;
    }
    return NAPSPMV_OK;
}

}  // extern "C"

// ===================================================================
// Batched CG steps over independent requests (the request server).
//
// Every slot is one CG solve with its own plan, vectors and scalars.  A dot
// product of slot i uses slot_blocks(n_i) blocks over a fixed strided
// partition of its own vectors and a fixed-order final sum: a function of its
// own length only, so its value does not depend on which other slots share
// the launch.  One block per 1,024 elements, at most 4,096; the final sum is
// one warp's, lanes over a fixed stride and a fixed shuffle tree.  A fixed 64
// blocks left a 1.7M-element solve latency-bound on its vector kernels (about
// 330 us per CG iteration on GB300).
namespace nap {
namespace {

constexpr int kMaxSlots = 64;
constexpr int kSlotBlocksMax = 4096;
constexpr int64_t kSlotChunk = 4 * 256;

__host__ __device__ __forceinline__ int slot_blocks(int64_t n)
{
    const int64_t b = (n + kSlotChunk - 1) / kSlotChunk;
    return (int)(b < 1 ? 1 : (b > kSlotBlocksMax ? kSlotBlocksMax : b));
}

enum Scl { S_RR = 0, S_PQ = 1, S_ALPHA = 2, S_BETA = 3, S_RRNEW = 4, S_BB = 5 };

struct SlotVecs {
    int32_t count;
    int64_t n[kMaxSlots];
    const double *b[kMaxSlots];
    double *x[kMaxSlots], *r[kMaxSlots], *p[kMaxSlots], *q[kMaxSlots], *scal[kMaxSlots];
};

__device__ __forceinline__ double block_sum_any(double v, double *sh)
{
    return block_sum(v, sh);
}

// mode 0: r = b - q, p = r, partial(r.r) and partial(b.b)
// mode 1: partial(p.q)
// mode 2: x += alpha p, r -= alpha q, partial(r.r)
// mode 3: p = r + beta p
// mode 4: r = b, p = b, partial(r.r), partial(b.b)   (x = 0)
__global__ void __launch_bounds__(kThreads) k_slot_vec(const __grid_constant__ SlotVecs S, int mode,
                                                       double *partial)
{
    __shared__ double sh[kThreads / 32];
    const int i = blockIdx.y;
    const int64_t n = S.n[i];
    const int nb = slot_blocks(n);
    if ((int)blockIdx.x >= nb) return;  // the whole block: this slot needs fewer
    const double *b = S.b[i];
    double *x = S.x[i], *r = S.r[i], *p = S.p[i], *q = S.q[i];
    const double alpha = mode == 2 ? S.scal[i][S_ALPHA] : 0.0;
    const double beta = mode == 3 ? S.scal[i][S_BETA] : 0.0;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < n;
         k += (int64_t)nb * kThreads) {
        if (mode == 0 || mode == 4) {
            const double v = mode == 0 ? b[k] - q[k] : b[k];
            r[k] = v;
            p[k] = v;
            if (mode == 4) x[k] = 0.0;
            s1 = fma(v, v, s1);
            s2 = fma(b[k], b[k], s2);
        } else if (mode == 1) {
            s1 = fma(p[k], q[k], s1);
        } else if (mode == 2) {
            x[k] = fma(alpha, p[k], x[k]);
            const double v = fma(-alpha, q[k], r[k]);
            r[k] = v;
            s1 = fma(v, v, s1);
        } else {
            p[k] = fma(beta, p[k], r[k]);
        }
    }
    if (mode == 3) return;
    s1 = block_sum_any(s1, sh);
    if (mode == 0 || mode == 4) s2 = block_sum_any(s2, sh);
    if (threadIdx.x == 0) {
        partial[((int64_t)i * kSlotBlocksMax + blockIdx.x) * 2 + 0] = s1;
        partial[((int64_t)i * kSlotBlocksMax + blockIdx.x) * 2 + 1] = s2;
    }
}

// Fixed-order sums of the partials (lane l adds partials l, l + 32, ... in
// order, then a fixed shuffle tree) and the scalar recurrences of CG.
__global__ void k_slot_final(const __grid_constant__ SlotVecs S, int mode, const double *partial)
{
    const int i = blockIdx.x, lane = threadIdx.x;
    double a = 0.0, c = 0.0;
    const int nb = slot_blocks(S.n[i]);
    for (int q = lane; q < nb; q += 32) {
        a += partial[((int64_t)i * kSlotBlocksMax + q) * 2 + 0];
        c += partial[((int64_t)i * kSlotBlocksMax + q) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane != 0) return;
    double *s = S.scal[i];
    if (mode == 0 || mode == 4) {
        s[S_RR] = a;
        s[S_BB] = c;
    } else if (mode == 1) {
        s[S_PQ] = a;
        s[S_ALPHA] = s[S_RR] / a;
    } else if (mode == 2) {
        s[S_RRNEW] = a;
        s[S_BETA] = a / s[S_RR];
        s[S_RR] = a;
    }
}

int slot_vec(const SlotVecs &S, int mode, double *partial, cudaStream_t st)
{
    int gx = 1;
    for (int i = 0; i < S.count; i++) gx = std::max(gx, slot_blocks(S.n[i]));
    k_slot_vec<<<dim3(gx, S.count), kThreads, 0, st>>>(S, mode, partial);
    count_launch(1);
    if (mode != 3) {
        k_slot_final<<<S.count, 32, 0, st>>>(S, mode, partial);
        count_launch(1);
    }
    NAP_CUDA(cudaGetLastError());
    return NAPSPMV_OK;
}

int slot_setup(int32_t count, const napspmv_cg_slot *slots, SlotVecs &S)
{
    if (count < 1 || count > kMaxSlots || !slots) {
        set_error(NAPSPMV_ERR_ARG, "need 1..64 CG slots");
        return NAPSPMV_ERR_ARG;
    }
    memset(&S, 0, sizeof(S));
    S.count = count;
    for (int i = 0; i < count; i++) {
        const napspmv_cg_slot &c = slots[i];
        if (!c.plan || !c.b || !c.x || !c.r || !c.p || !c.q || !c.scal) {
            set_error(NAPSPMV_ERR_ARG, "CG slot with a NULL pointer");
            return NAPSPMV_ERR_ARG;
        }
        S.n[i] = c.plan->n;
        S.b[i] = c.b;
        S.x[i] = c.x;
        S.r[i] = c.r;
        S.p[i] = c.p;
        S.q[i] = c.q;
        S.scal[i] = c.scal;
    }
    return NAPSPMV_OK;
}

int slot_apply(int32_t count, const napspmv_cg_slot *slots, bool from_x, int32_t precision,
               cudaStream_t st)
{
    napspmv_plan_t *plans[kMaxSlots];
    napspmv_ws_t *wss[kMaxSlots];
    const double *vs[kMaxSlots];
    double *ws_[kMaxSlots];
    int32_t reps[kMaxSlots];
    double sc[kMaxSlots];
    for (int i = 0; i < count; i++) {
        plans[i] = slots[i].plan;
        wss[i] = slots[i].ws;
        vs[i] = from_x ? slots[i].x : slots[i].p;
        ws_[i] = slots[i].q;
        reps[i] = 1;
        sc[i] = 1.0;
    }
    // A slot whose matrix holds NAPSPMV_SOLO_NNZ or more stored entries gets an
    // apply of its own on the phased engine; the others share one persistent
    // launch.  Measured on GB300 (FP32 mode, one apply): a 2.0M-row 7-point
    // plan takes 77 us phased against 191 us in the persistent launch, a
    // 0.4M-row one 33 against 70 us; below about half a million entries the
    // shared launch costs less than a call per slot.  The choice depends on the
    // slot's own matrix only, and every slot runs with its own plan's default
    // options (slots whose defaults differ go into separate fused launches), so
    // a slot's bits do not depend on the batch.
    int nb = 0;
    for (int i = 0; i < count; i++) {
        if (plans[i]->nnz >= NAPSPMV_SOLO_NNZ) {
            napspmv_opts o = plans[i]->defaults;
            o.precision = precision;
            o.engine = NAPSPMV_ENGINE_PHASED;
            if (int rc = apply_batch(1, &plans[i], &wss[i], &vs[i], &ws_[i], &reps[i], &sc[i], &o, st))
                return rc;
        } else {
            plans[nb] = plans[i];
            wss[nb] = wss[i];
            vs[nb] = vs[i];
            ws_[nb] = ws_[i];
            nb++;
        }
    }
    if (nb == 0) return NAPSPMV_OK;
    napspmv_opts o{};  // unset fields: each slot's own plan defaults
    o.precision = precision;
    o.engine = NAPSPMV_ENGINE_FUSED;
    return apply_batch(nb, plans, wss, vs, ws_, reps, sc, &o, st);
}

struct Partials {
    double *p = nullptr;
    cudaStream_t s = 0;
    ~Partials()
    {
        if (p) cudaFreeAsync(p, s);
    }
};

}  // namespace
}  // namespace nap

extern "C" {

int napspmv_cg_batch_init(int32_t count, const napspmv_cg_slot *slots, int32_t precision,
                          int32_t x_is_zero, void *stream)
{
    SlotVecs S;
    int rc = slot_setup(count, slots, S);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Partials P;
    P.s = st;
    NAP_CUDA(cudaMallocAsync(&P.p, sizeof(double) * 2 * kSlotBlocksMax * count, st));
    if (x_is_zero) return slot_vec(S, 4, P.p, st);
    if ((rc = slot_apply(count, slots, true, precision, st))) return rc;
    return slot_vec(S, 0, P.p, st);
}

int napspmv_cg_batch_iterate(int32_t count, const napspmv_cg_slot *slots, int32_t precision,
                             int32_t iters, void *stream)
{
    SlotVecs S;
    int rc = slot_setup(count, slots, S);
    if (rc) return rc;
    if (iters < 0) {
        set_error(NAPSPMV_ERR_ARG, "iters < 0");
        return NAPSPMV_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Partials P;
    P.s = st;
    NAP_CUDA(cudaMallocAsync(&P.p, sizeof(double) * 2 * kSlotBlocksMax * count, st));
    for (int it = 0; it < iters; it++) {
        if ((rc = slot_apply(count, slots, false, precision, st))) return rc;
        if ((rc = slot_vec(S, 1, P.p, st))) return rc;
        if ((rc = slot_vec(S, 2, P.p, st))) return rc;
        if ((rc = slot_vec(S, 3, P.p, st))) return rc;
    }
    return NAPSPMV_OK;
}

}  // extern "C"

namespace nap {
namespace {
struct AddVecs {
    int32_t count;
    int64_t n[kMaxSlots];
    double *y[kMaxSlots];
    const double *x[kMaxSlots];
};
__global__ void k_slot_add(const __grid_constant__ AddVecs A)
{
    const int i = blockIdx.y;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < A.n[i];
         k += (int64_t)gridDim.x * blockDim.x)
        A.y[i][k] += A.x[i][k];
}
}  // namespace
}  // namespace nap

extern "C" int napspmv_batch_add(int32_t count, double *const *y, const double *const *x,
                                 const int64_t *n, void *stream)
{
    if (count < 1 || count > kMaxSlots || !y || !x || !n) {
        set_error(NAPSPMV_ERR_ARG, "need 1..64 vector pairs");
        return NAPSPMV_ERR_ARG;
    }
    AddVecs A;
    memset(&A, 0, sizeof(A));
    A.count = count;
    for (int i = 0; i < count; i++) {
        if (!y[i] || !x[i] || n[i] < 0) {
            set_error(NAPSPMV_ERR_ARG, "NULL vector or n < 0");
            return NAPSPMV_ERR_ARG;
        }
        A.y[i] = y[i];
        A.x[i] = x[i];
        A.n[i] = n[i];
    }
    int gx = 1;
    for (int i = 0; i < count; i++) gx = std::max(gx, slot_blocks(n[i]));
    k_slot_add<<<dim3(gx, count), kThreads, 0, (cudaStream_t)stream>>>(A);
    count_launch(1);
    NAP_CUDA(cudaGetLastError());
    return NAPSPMV_OK;
}
