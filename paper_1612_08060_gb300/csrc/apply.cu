// apply.cu -- the node-aware SpMV apply on one GPU.
//
// Algorithm NAPSpMV (Sec. 4) with local_comm (Sec. 4.2) for all simulated
// processes at once.  Every message becomes a device gather or copy in HBM:
//
//   phase 1  on_node -> on_node   b_{l->l}[k]  = x[bll_j[k]]       (Eq. IL2)
//            on_node -> off_node  b_{l->nl}[k] = x[lbuf_j[k]]      (Eq. IL0)
//   phase 2  pack g_send from x (own values) or b_{l->nl}          (Eq. I)
//   phase 3  inter-node transfer g_send -> g_recv (the "network")
//   phase 4  off_node -> on_node  b_{nl->l}[k] = g_recv[unp_src[k]] (Eq. IL1)
//   phase 5  three-block SpMV: on_process from x, on_node from b_{l->l},
//            off_node from b_{nl->l} (three local_spmv of the algorithm in one
//            pass over each row)
//
// Fused engine: one persistent launch.  CTAs take work items (chunks of a
// node's gather ranges, tiles of a node's rows) from a global ticket counter
// in topological order; before an item runs, thread 0 waits (bounded, with a
// device error flag on timeout) on per-node counters of the items it depends
// on, so node n's SpMV starts as soon as node n's buffers are complete and a
// chain of applies x_{k+1} = scale A x_k pipelines across nodes.  Tickets are
// handed out in order and an item only waits on earlier tickets, so progress
// never depends on how many CTAs are resident.
//
// Phased engine (control): one kernel per phase per apply.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace nap {

// ------------------------------------------------------------ error state
static thread_local std::string g_last_error;
static thread_local int64_t g_launches = 0;

void set_error(int code, const std::string &msg)
{
    g_last_error = std::string(napspmv_strerror(code)) + ": " + msg;
}
int cuda_error(cudaError_t e, const char *what)
{
    cudaGetLastError();
    int code = e == cudaErrorMemoryAllocation ? NAPSPMV_ERR_OOM : NAPSPMV_ERR_CUDA;
    set_error(code, std::string(what) + ": " + cudaGetErrorString(e));
    return code;
}
void count_launch(int64_t n) { g_launches += n; }

// ---------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_stream_s32(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream_f64(const double *p)
{
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream_f32(const float *p)
{
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long globaltimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Vector loads: data written earlier in the same launch is read through L2
// (L1 is not coherent across SMs); in the phased engine every vector is
// read-only for the kernel's lifetime and may use the read-only path.
template <bool INKERNEL>
__device__ __forceinline__ double ldx(const double *p)
{
    if (INKERNEL) return __ldcg(p);
    return __ldg(p);
}

// ------------------------------------------------------- three-block SpMV
struct Csr3 {
    const int32_t *rowptr;
    const uint32_t *colenc;
    const double *val;
    const float *val32;
};

// Rows [r0, r1): V lanes per row, 256 threads.  All lanes of a warp run the
// same number of outer iterations, so the shuffle reduction is convergent.
template <int V, bool F32, bool INKERNEL>
__device__ __forceinline__ void spmv_rows(const Csr3 &A, const double *x, const double *bll,
                                          const double *bnl, double *y, double scale, int r0,
                                          int r1, int tid, int nthreads)
{
    const int lane = tid & (V - 1);
    const int grp = tid / V;
    const int groups = nthreads / V;
    for (int base = r0; base < r1; base += groups) {
        const int row = base + grp;
        double acc = 0.0;
        if (row < r1) {
            const int s = ld_stream_s32(A.rowptr + row), e = ld_stream_s32(A.rowptr + row + 1);
#pragma unroll 2
            for (int k = s + lane; k < e; k += V) {
                const uint32_t c = ld_stream_u32(A.colenc + k);
                const uint32_t blk = c >> kBlockShift;
                const double *src = blk == 0 ? x : (blk == 1 ? bll : bnl);
                const double xv = ldx<INKERNEL>(src + (c & kIndexMask));
                if (F32) {
                    const float a = ld_stream_f32(A.val32 + k);
                    const float p = __fmul_rn(a, __double2float_rn(xv));
                    acc = __dadd_rn(acc, (double)p);
                } else {
                    acc = fma(ld_stream_f64(A.val + k), xv, acc);
                }
            }
        }
        if (V > 1) {
#pragma unroll
            for (int o = V / 2; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        }
        if (row < r1 && lane == 0) y[row] = scale == 1.0 ? acc : scale * acc;
    }
}

// ---------------------------------------------------------- fused engine
struct Job {
    const Item *items;
    int32_t n_items;
    int32_t reps;
    double scale;
    long long tbase;  // first ticket of this job in the launch
    Csr3 A;
    const int32_t *bll_j, *lbuf_j, *xfer_dst, *unp_src;
    const uint32_t *pack_src;
    const int32_t *msg_off, *msg_dstnode;
    const uint64_t *cnt;  // [kNumCounters][nn] per-apply increments
    int32_t nn;
    double *bll, *lbuf, *gsend, *grecv, *bnl, *xtmp;
    unsigned long long *ctr;  // [0] ticket, then [kNumCounters][nn], then one spare
    int *err;
    const double *v;
    double *w;
};

template <int MAXJ>
struct FusedParams {
    int32_t njobs;
    int32_t stall;
    long long total;
    long long timeout_ns;
    unsigned long long *ticket;
    Job jobs[MAXJ];
};

__device__ __forceinline__ bool wait_ge(const unsigned long long *p, unsigned long long target,
                                        int *err, long long timeout_ns)
{
    if (target == 0 || ld_acquire(p) >= target) return true;
    const long long t0 = globaltimer();
    unsigned ns = 64;
    for (;;) {
        if (*(volatile int *)err) return false;
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
        if (ld_acquire(p) >= target) return true;
        if (globaltimer() - t0 > timeout_ns) {
            atomicCAS(err, 0, 1);
            return false;
        }
    }
}

__device__ bool item_deps(const Job &J, const Item &it, int k, long long tmo, bool stall)
{
    auto C = [&](int c, int node) { return J.ctr + 1 + c * J.nn + node; };
    auto N = [&](int c, int node) { return (unsigned long long)J.cnt[c * J.nn + node]; };
    const unsigned long long kk = k, k1 = k + 1;
    const int n = it.node;
    if (stall && !wait_ge(J.ctr + 1 + kNumCounters * J.nn, 1, J.err, tmo)) return false;
    switch (it.kind) {
    case kGatherJ2:
    case kGatherJ0:
        // x_k rows of node n written; previous readers of b_{l->l}, b_{l->nl} done
        return wait_ge(C(kC5, n), kk * N(kC5, n), J.err, tmo) &&
               wait_ge(C(kC2, n), kk * N(kC2, n), J.err, tmo);
    case kPack:
        return wait_ge(C(kC1, n), k1 * N(kC1, n), J.err, tmo) &&
               wait_ge(C(kC5, n), kk * N(kC5, n), J.err, tmo) &&
               wait_ge(C(kC3, n), kk * N(kC3, n), J.err, tmo);
    case kTransfer: {
        if (!wait_ge(C(kC2, n), k1 * N(kC2, n), J.err, tmo)) return false;
        if (k == 0) return true;
        for (int m = it.msg; J.msg_off[m] < it.e; m++) {
            const int dn = J.msg_dstnode[m];
            if (!wait_ge(C(kC4, dn), kk * N(kC4, dn), J.err, tmo)) return false;
        }
        return true;
    }
    case kUnpack:
        return wait_ge(C(kArr, n), k1 * N(kArr, n), J.err, tmo) &&
               wait_ge(C(kC5, n), kk * N(kC5, n), J.err, tmo);
    default:  // kSpmv
        return wait_ge(C(kC1, n), k1 * N(kC1, n), J.err, tmo) &&
               wait_ge(C(kC4, n), k1 * N(kC4, n), J.err, tmo) &&
               wait_ge(C(kC5, n), kk * N(kC5, n), J.err, tmo) &&
               wait_ge(C(kC2, n), kk * N(kC2, n), J.err, tmo);
    }
}

__device__ void item_signal(const Job &J, const Item &it)
{
    auto C = [&](int c, int node) { return J.ctr + 1 + c * J.nn + node; };
    switch (it.kind) {
    case kGatherJ2:
    case kGatherJ0: atomicAdd(C(kC1, it.node), 1ull); break;
    case kPack: atomicAdd(C(kC2, it.node), 1ull); break;
    case kTransfer:
        for (int m = it.msg; J.msg_off[m] < it.e; m++) {
            const int lo = max(it.b, J.msg_off[m]), hi = min(it.e, J.msg_off[m + 1]);
            if (hi > lo) atomicAdd(C(kArr, J.msg_dstnode[m]), (unsigned long long)(hi - lo));
        }
        atomicAdd(C(kC3, it.node), 1ull);
        break;
    case kUnpack: atomicAdd(C(kC4, it.node), 1ull); break;
    default: atomicAdd(C(kC5, it.node), 1ull); break;
    }
}

template <int V, bool F32, int MAXJ>
__global__ void __launch_bounds__(256) k_fused(const __grid_constant__ FusedParams<MAXJ> prm)
{
    __shared__ long long s_t;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_t = (long long)atomicAdd(prm.ticket, 1ull);
        __syncthreads();
        const long long t = s_t;
        if (t >= prm.total) break;
        int ji = 0;
        while (ji + 1 < prm.njobs && prm.jobs[ji + 1].tbase <= t) ji++;
        const Job &J = prm.jobs[ji];
        const long long tl = t - J.tbase;
        const int k = (int)(tl / J.n_items);
        const Item it = J.items[tl % J.n_items];
        // a sticky error (an earlier wait timed out) stops all work of the job
        if (tid == 0)
            s_ok = !*(volatile int *)J.err && item_deps(J, it, k, prm.timeout_ns, prm.stall && t == 0);
        __syncthreads();
        if (!s_ok) break;
        const double *x = (k == 0) ? J.v : (((J.reps - k) & 1) == 0 ? J.w : J.xtmp);
        double *y = (((J.reps - 1 - k) & 1) == 0) ? J.w : J.xtmp;
        switch (it.kind) {
        case kGatherJ2:
            for (int e = it.b + tid; e < it.e; e += 256) J.bll[e] = __ldcg(x + ld_stream_s32(J.bll_j + e));
            break;
        case kGatherJ0:
            for (int e = it.b + tid; e < it.e; e += 256) J.lbuf[e] = __ldcg(x + ld_stream_s32(J.lbuf_j + e));
            break;
        case kPack:
            for (int e = it.b + tid; e < it.e; e += 256) {
                const uint32_t u = ld_stream_u32(J.pack_src + e);
                J.gsend[e] = (u & kFromLbuf) ? __ldcg(J.lbuf + (u & ~kFromLbuf)) : __ldcg(x + u);
            }
            break;
        case kTransfer:
            for (int e = it.b + tid; e < it.e; e += 256) J.grecv[ld_stream_s32(J.xfer_dst + e)] = __ldcg(J.gsend + e);
            break;
        case kUnpack:
            for (int e = it.b + tid; e < it.e; e += 256) J.bnl[e] = __ldcg(J.grecv + ld_stream_s32(J.unp_src + e));
            break;
        default:
            spmv_rows<V, F32, true>(J.A, x, J.bll, J.bnl, y, J.scale, it.b, it.e, tid, 256);
            break;
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            item_signal(J, it);
        }
    }
}

// --------------------------------------------------------- phased engine
__global__ void k_gather2(const double *__restrict__ x, const int32_t *__restrict__ bll_j,
                          double *__restrict__ bll, int n_bll, const int32_t *__restrict__ lbuf_j,
                          double *__restrict__ lbuf, int n_lbuf)
{
    const int total = n_bll + n_lbuf;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        if (e < n_bll)
            bll[e] = __ldg(x + ld_stream_s32(bll_j + e));
        else
            lbuf[e - n_bll] = __ldg(x + ld_stream_s32(lbuf_j + e - n_bll));
    }
}
__global__ void k_pack(const double *__restrict__ x, const double *__restrict__ lbuf,
                       const uint32_t *__restrict__ src, double *__restrict__ gsend, int n)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t u = ld_stream_u32(src + e);
        gsend[e] = (u & kFromLbuf) ? __ldg(lbuf + (u & ~kFromLbuf)) : __ldg(x + u);
    }
}
__global__ void k_transfer(const double *__restrict__ gsend, const int32_t *__restrict__ dst,
                           double *__restrict__ grecv, int n)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        grecv[ld_stream_s32(dst + e)] = __ldg(gsend + e);
}
__global__ void k_unpack(const double *__restrict__ grecv, const int32_t *__restrict__ src,
                         double *__restrict__ bnl, int n)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        bnl[e] = __ldg(grecv + ld_stream_s32(src + e));
}
template <int V, bool F32>
__global__ void __launch_bounds__(256) k_spmv(Csr3 A, const double *x, const double *bll,
                                              const double *bnl, double *y, double scale, int n,
                                              int rows_per_block)
{
    for (int r0 = blockIdx.x * rows_per_block; r0 < n; r0 += gridDim.x * rows_per_block)
        spmv_rows<V, F32, false>(A, x, bll, bnl, y, scale, r0, min(n, r0 + rows_per_block),
                                 threadIdx.x, 256);
}

// ------------------------------------------------------------- dispatch
template <int MAXJ>
struct FusedKernelTable {
    using Fn = void (*)(const FusedParams<MAXJ>);
    static Fn get(int vec, bool f32)
    {
#define NAP_CASE(V)                                                   \
    case V: return f32 ? k_fused<V, true, MAXJ> : k_fused<V, false, MAXJ>;
        switch (vec) {
            NAP_CASE(1)
            NAP_CASE(2)
            NAP_CASE(4)
            NAP_CASE(8)
            NAP_CASE(16)
            NAP_CASE(32)
        }
#undef NAP_CASE
        return nullptr;
    }
};

static bool valid_vec(int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32; }

napspmv_opts resolve_opts(const napspmv_plan_t *P, const napspmv_opts *o)
{
    napspmv_opts r = P->defaults;
    if (!o) return r;
    r.precision = o->precision;  // 0 is FP64, a real choice
    r.engine = o->engine;
    if (o->vec) r.vec = o->vec;
    if (o->ctas_per_sm) r.ctas_per_sm = o->ctas_per_sm;
    if (o->chunk) r.chunk = o->chunk;
    if (o->tile_rows) r.tile_rows = o->tile_rows;
    if (o->timeout_ms) r.timeout_ms = o->timeout_ms;
    r.debug_stall = o->debug_stall;
    return r;
}

int build_items(napspmv_plan_t *P, int32_t chunk, int32_t tile_rows)
{
    if (chunk < 32 || tile_rows < 1) {
        set_error(NAPSPMV_ERR_ARG, "chunk must be >= 32 and tile_rows >= 1");
        return NAPSPMV_ERR_ARG;
    }
    ItemSet &S = P->items;
    if (S.d_items && S.chunk == chunk && S.tile_rows == tile_rows) return NAPSPMV_OK;
    const int nn = P->nn;
    std::vector<Item> items;
    std::vector<uint64_t> cnt((size_t)kNumCounters * nn, 0);
    auto add = [&](int kind, int node, int64_t b, int64_t e, int msg, int counter) {
        Item it{};
        it.kind = kind;
        it.node = node;
        it.b = (int32_t)b;
        it.e = (int32_t)e;
        it.msg = msg;
        items.push_back(it);
        cnt[(size_t)counter * nn + node]++;
    };
    for (int x = 0; x < nn; x++)
        for (int64_t b = P->node_bll[x]; b < P->node_bll[x + 1]; b += chunk)
            add(kGatherJ2, x, b, std::min<int64_t>(b + chunk, P->node_bll[x + 1]), 0, kC1);
    for (int x = 0; x < nn; x++)
        for (int64_t b = P->node_lbuf[x]; b < P->node_lbuf[x + 1]; b += chunk)
            add(kGatherJ0, x, b, std::min<int64_t>(b + chunk, P->node_lbuf[x + 1]), 0, kC1);
    for (int x = 0; x < nn; x++)
        for (int64_t b = P->node_gs[x]; b < P->node_gs[x + 1]; b += chunk)
            add(kPack, x, b, std::min<int64_t>(b + chunk, P->node_gs[x + 1]), 0, kC2);
    const std::vector<int64_t> &off = P->gs_msg_off;
    for (int x = 0; x < nn; x++)
        for (int64_t b = P->node_gs[x]; b < P->node_gs[x + 1]; b += chunk) {
            int m = (int)(std::upper_bound(off.begin(), off.end(), b) - off.begin()) - 1;
            add(kTransfer, x, b, std::min<int64_t>(b + chunk, P->node_gs[x + 1]), m, kC3);
        }
    for (size_t m = 0; m + 1 < off.size(); m++)
        cnt[(size_t)kArr * nn + P->gs_msg_dstnode[m]] += (uint64_t)(off[m + 1] - off[m]);
    for (int x = 0; x < nn; x++)
        for (int64_t b = P->node_bnl[x]; b < P->node_bnl[x + 1]; b += chunk)
            add(kUnpack, x, b, std::min<int64_t>(b + chunk, P->node_bnl[x + 1]), 0, kC4);
    for (int x = 0; x < nn; x++)
        for (int64_t b = P->node_rows[x]; b < P->node_rows[x + 1]; b += tile_rows)
            add(kSpmv, x, b, std::min<int64_t>(b + tile_rows, P->node_rows[x + 1]), 0, kC5);

    Item *d_items = nullptr;
    uint64_t *d_cnt = nullptr;
    NAP_CUDA(cudaMalloc(&d_items, sizeof(Item) * items.size()));
    NAP_CUDA(cudaMalloc(&d_cnt, sizeof(uint64_t) * cnt.size()));
    NAP_CUDA(cudaMemcpy(d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice));
    NAP_CUDA(cudaMemcpy(d_cnt, cnt.data(), sizeof(uint64_t) * cnt.size(), cudaMemcpyHostToDevice));
    if (S.d_items) cudaFree(S.d_items);
    if (S.d_cnt) cudaFree(S.d_cnt);
    S.d_items = d_items;
    S.d_cnt = d_cnt;
    S.n_items = (int32_t)items.size();
    S.chunk = chunk;
    S.tile_rows = tile_rows;
    return NAPSPMV_OK;
}

static size_t ctr_count(const napspmv_plan_t *P) { return 2 + (size_t)kNumCounters * P->nn; }

int ws_alloc(napspmv_plan_t *P, napspmv_ws_t *ws)
{
    ws->plan = P;
    ws->device = P->device;
    auto al = [](double **p, int64_t n) {
        return cudaMalloc(p, sizeof(double) * (size_t)std::max<int64_t>(n, 1));
    };
    if (al(&ws->bll, P->n_bll) || al(&ws->lbuf, P->n_lbuf) || al(&ws->gsend, P->n_gs) ||
        al(&ws->grecv, P->n_gs) || al(&ws->bnl, P->n_bnl) || al(&ws->xtmp, P->n) ||
        cudaMalloc(&ws->ctr, sizeof(unsigned long long) * ctr_count(P)) ||
        cudaMalloc(&ws->err, sizeof(int))) {
        ws_free(ws);
        return cuda_error(cudaErrorMemoryAllocation, "workspace");
    }
    if (cudaMemset(ws->err, 0, sizeof(int)) != cudaSuccess) {
        ws_free(ws);
        return cuda_error(cudaGetLastError(), "workspace");
    }
    return NAPSPMV_OK;
}

void ws_free(napspmv_ws_t *ws)
{
    void *p[] = {ws->bll, ws->lbuf, ws->gsend, ws->grecv, ws->bnl, ws->xtmp, ws->hv, ws->hw,
                 ws->ctr, ws->err};
    for (void *q : p)
        if (q) cudaFree(q);
    ws->bll = ws->lbuf = ws->gsend = ws->grecv = ws->bnl = ws->xtmp = ws->hv = ws->hw = nullptr;
    ws->ctr = nullptr;
    ws->err = nullptr;
}

static Job make_job(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w, int reps,
                    double scale, bool f32)
{
    Job J{};
    J.items = P->items.d_items;
    J.n_items = P->items.n_items;
    J.reps = reps;
    J.scale = scale;
    J.A = Csr3{P->d_rowptr, P->d_colenc, P->d_val, f32 ? P->d_val32 : nullptr};
    J.bll_j = P->lists[L_BLL].d_idx;
    J.lbuf_j = P->lists[L_LBUF].d_idx;
    J.xfer_dst = P->d_xfer_dst;
    J.unp_src = P->d_unp_src;
    J.pack_src = P->d_pack_src;
    J.msg_off = P->d_gs_msg_off;
    J.msg_dstnode = P->d_gs_msg_dstnode;
    J.cnt = P->items.d_cnt;
    J.nn = P->nn;
    J.bll = ws->bll;
    J.lbuf = ws->lbuf;
    J.gsend = ws->gsend;
    J.grecv = ws->grecv;
    J.bnl = ws->bnl;
    J.xtmp = ws->xtmp;
    J.ctr = ws->ctr;
    J.err = ws->err;
    J.v = v;
    J.w = w;
    return J;
}

template <int MAXJ>
static int launch_fused(int count, napspmv_plan_t *const *plans, napspmv_ws_t *const *ws,
                        const double *const *v, double *const *w, const int32_t *reps,
                        const double *scale, const napspmv_opts &o, cudaStream_t s)
{
    FusedParams<MAXJ> prm;
    memset(&prm, 0, sizeof(prm));
    prm.njobs = count;
    prm.stall = o.debug_stall ? 1 : 0;
    prm.timeout_ns = (long long)o.timeout_ms * 1000000ll;
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    long long total = 0;
    for (int i = 0; i < count; i++) {
        napspmv_ws_t *wi = ws && ws[i] ? ws[i] : plans[i]->ws;
        prm.jobs[i] = make_job(plans[i], wi, v[i], w[i], reps[i], scale ? scale[i] : 1.0, f32);
        prm.jobs[i].tbase = total;
        total += (long long)prm.jobs[i].n_items * reps[i];
        NAP_CUDA(cudaMemsetAsync(wi->ctr, 0, sizeof(unsigned long long) * ctr_count(plans[i]), s));
    }
    prm.total = total;
    prm.ticket = prm.jobs[0].ctr;
    auto fn = FusedKernelTable<MAXJ>::get(o.vec, f32);
    int occ = 0;
    NAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0));
    int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, std::max(occ, 1)) : std::max(occ, 1);
    long long grid = (long long)plans[0]->num_sms * per_sm;
    grid = std::max(1ll, std::min(grid, total));
    fn<<<(int)grid, 256, 0, s>>>(prm);
    NAP_CUDA(cudaGetLastError());
    count_launch(1);
    return NAPSPMV_OK;
}

static int launch_phased(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w, int reps,
                         double scale, const napspmv_opts &o, cudaStream_t s)
{
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    const int T = 256;
    auto grid = [&](int64_t n) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((n + T - 1) / T, (int64_t)P->num_sms * 8));
    };
    Csr3 A{P->d_rowptr, P->d_colenc, P->d_val, f32 ? P->d_val32 : nullptr};
    using SpmvFn = void (*)(Csr3, const double *, const double *, const double *, double *, double,
                            int, int);
    SpmvFn sp = nullptr;
#define NAP_CASE(V) \
    case V: sp = f32 ? k_spmv<V, true> : k_spmv<V, false>; break;
    switch (o.vec) {
        NAP_CASE(1)
        NAP_CASE(2)
        NAP_CASE(4)
        NAP_CASE(8)
        NAP_CASE(16)
        NAP_CASE(32)
    }
#undef NAP_CASE
    const int rows_per_block = 256 / o.vec * 4;
    for (int k = 0; k < reps; k++) {
        const double *x = (k == 0) ? v : (((reps - k) & 1) == 0 ? w : ws->xtmp);
        double *y = (((reps - 1 - k) & 1) == 0) ? w : ws->xtmp;
        if (P->n_bll + P->n_lbuf > 0) {
            k_gather2<<<grid(P->n_bll + P->n_lbuf), T, 0, s>>>(x, P->lists[L_BLL].d_idx, ws->bll,
                                                               (int)P->n_bll, P->lists[L_LBUF].d_idx,
                                                               ws->lbuf, (int)P->n_lbuf);
            count_launch(1);
        }
        if (P->n_gs > 0) {
            k_pack<<<grid(P->n_gs), T, 0, s>>>(x, ws->lbuf, P->d_pack_src, ws->gsend, (int)P->n_gs);
            k_transfer<<<grid(P->n_gs), T, 0, s>>>(ws->gsend, P->d_xfer_dst, ws->grecv, (int)P->n_gs);
            count_launch(2);
        }
        if (P->n_bnl > 0) {
            k_unpack<<<grid(P->n_bnl), T, 0, s>>>(ws->grecv, P->d_unp_src, ws->bnl, (int)P->n_bnl);
            count_launch(1);
        }
        const int64_t nb = (P->n + rows_per_block - 1) / rows_per_block;
        sp<<<(int)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)P->num_sms * 16)), T, 0, s>>>(
            A, x, ws->bll, ws->bnl, y, scale, (int)P->n, rows_per_block);
        count_launch(1);
        NAP_CUDA(cudaGetLastError());
    }
    return NAPSPMV_OK;
}

static int check_opts(const napspmv_plan_t *P, const napspmv_opts &o)
{
    if (!valid_vec(o.vec)) {
        set_error(NAPSPMV_ERR_ARG, "vec must be 1, 2, 4, 8, 16 or 32");
        return NAPSPMV_ERR_ARG;
    }
    if (o.precision != NAPSPMV_PREC_F64 && o.precision != NAPSPMV_PREC_F32) {
        set_error(NAPSPMV_ERR_ARG, "unknown precision");
        return NAPSPMV_ERR_ARG;
    }
    if (o.precision == NAPSPMV_PREC_F32 && !P->d_val32) {
        set_error(NAPSPMV_ERR_STATE, "plan was built without NAPSPMV_F32_VALUES");
        return NAPSPMV_ERR_STATE;
    }
    if (o.engine != NAPSPMV_ENGINE_FUSED && o.engine != NAPSPMV_ENGINE_PHASED) {
        set_error(NAPSPMV_ERR_ARG, "unknown engine");
        return NAPSPMV_ERR_ARG;
    }
    if (o.timeout_ms < 1) {
        set_error(NAPSPMV_ERR_ARG, "timeout_ms must be >= 1");
        return NAPSPMV_ERR_ARG;
    }
    return NAPSPMV_OK;
}

int apply_batch(int32_t count, napspmv_plan_t *const *plans, napspmv_ws_t *const *ws,
                const double *const *v, double *const *w, const int32_t *reps, const double *scale,
                const napspmv_opts *opts, cudaStream_t s)
{
    if (count < 1 || count > 64 || !plans || !v || !w || !reps) {
        set_error(NAPSPMV_ERR_ARG, "batch needs 1..64 entries and non-NULL arrays");
        return NAPSPMV_ERR_ARG;
    }
    napspmv_plan_t *P0 = plans[0];
    if (!P0) {
        set_error(NAPSPMV_ERR_ARG, "NULL plan");
        return NAPSPMV_ERR_ARG;
    }
    napspmv_opts o = resolve_opts(P0, opts);
    for (int i = 0; i < count; i++) {
        napspmv_plan_t *P = plans[i];
        if (!P || !v[i] || !w[i] || reps[i] < 1 || (const double *)w[i] == v[i]) {
            set_error(NAPSPMV_ERR_ARG, "NULL plan or vector, reps < 1, or w == v");
            return NAPSPMV_ERR_ARG;
        }
        if (P->device != P0->device) {
            set_error(NAPSPMV_ERR_ARG, "all plans of a batch must live on one device");
            return NAPSPMV_ERR_ARG;
        }
        int rc = check_opts(P, o);
        if (rc) return rc;
        if (count > 1 || o.engine == NAPSPMV_ENGINE_FUSED) {
            rc = build_items(P, o.chunk, o.tile_rows);
            if (rc) return rc;
        }
        for (int q = 0; q < i; q++) {
            napspmv_ws_t *a = ws && ws[i] ? ws[i] : P->ws;
            napspmv_ws_t *b = ws && ws[q] ? ws[q] : plans[q]->ws;
            if (a == b) {
                set_error(NAPSPMV_ERR_ARG, "two batch entries share one workspace");
                return NAPSPMV_ERR_ARG;
            }
        }
        if (ws && ws[i] && ws[i]->plan != P) {
            set_error(NAPSPMV_ERR_ARG, "workspace belongs to another plan");
            return NAPSPMV_ERR_ARG;
        }
    }
    int cur = 0;
    NAP_CUDA(cudaGetDevice(&cur));
    if (cur != P0->device) NAP_CUDA(cudaSetDevice(P0->device));
    int rc;
    if (count == 1 && o.engine == NAPSPMV_ENGINE_PHASED)
        rc = launch_phased(P0, ws && ws[0] ? ws[0] : P0->ws, v[0], w[0], reps[0],
                           scale ? scale[0] : 1.0, o, s);
    else if (count == 1)
        rc = launch_fused<1>(count, plans, ws, v, w, reps, scale, o, s);
    else
        rc = launch_fused<64>(count, plans, ws, v, w, reps, scale, o, s);
    if (cur != P0->device) cudaSetDevice(cur);
    return rc;
}

}  // namespace nap

extern "C" const char *napspmv_last_error(void) { return nap::g_last_error.c_str(); }
extern "C" int64_t napspmv_launch_count(void) { return nap::g_launches; }
