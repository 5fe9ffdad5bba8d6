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
//            off_node from b_{nl->l} (the three local_spmv of the algorithm as
//            one pass over each row, blocks in that order)
//
// SpMV pipelines: sliced rows (rows sorted by length, 32 to a chunk,
// column-major, one lane per row, no shared-memory stage; the default for rows
// of more than 12 entries and the fused engine's), and CTA or warp row tiles.
// A row tile: one thread copies the tile's row-pointer, column and value slices
// into a shared-memory stage with bulk asynchronous copies counted on an
// mbarrier; the next tile's copy overlaps the current tile.  Each row is then
// summed from shared memory by one lane (vec lanes for long rows) with x and
// the receive buffers gathered from L2/HBM: one DFMA per stored entry (FP64
// issue, not only HBM, bounds the SpMV on GB300).  Stages are sized to each
// tile list's largest tile; tiles are handed to CTAs in contiguous runs.
//
// Engines:
//   overlapped (default for rows of at most 12 entries)  the matrix split into
//       its on_process part (local, needs no message) and its remote part; the
//       local pass runs on a second stream while the message steps run, the
//       remote pass continues each row's FMA chain from the local partial.
//       Where remote rows are gather-heavy, the remote pass stages each
//       process's receive buffers in shared memory.
//   phased (default for longer rows)  one kernel per phase per apply with the
//       single-pass SpMV.
//   fused    one persistent, cooperative launch for all phases and applies of
//       one or more jobs, in levels separated by bounded grid barriers (see
//       k_fused).  It also runs batches of independent applies in one launch.
// The phased engines capture chained applies into CUDA graphs and launch
// dependent kernels programmatically (resident while the predecessor drains).
// With one lane per row every engine gives the same bits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

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

constexpr int NT = 256;  // threads per CTA of every apply kernel

// ---------------------------------------------------------- PTX helpers
// Read-only streams (matrix, index arrays): non-coherent path, no L1 allocation.
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_stream_s32(const int32_t *p)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream_f64(const double *p)
{
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream_f32(const float *p)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
// L2 cache policies: streams read once (matrix, index arrays) are evicted
// first, so the gathered vectors (v, b_{l->l}, b_{nl->l}) stay L2-resident.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double ld_keep_f64(const double *p, uint64_t pol)
{
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream_hint_s32(const int32_t *p, uint64_t pol)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_hint_u32(const uint32_t *p, uint64_t pol)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic-serialization attribute may become resident while its
// predecessor in the stream drains: griddep_wait() waits, in hardware, until
// the predecessor grid has completed and its writes are visible, and
// griddep_done(), called when a CTA has issued its last work, lets the
// dependent grid start as this grid's CTAs finish (a CTA that exits early
// counts as done).  Without a programmatic predecessor both are no-ops.
__device__ __forceinline__ void griddep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_done()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ long long globaltimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Vector loads.  Fused engine: data written earlier in the same launch by
// other CTAs is read with plain (weak, L1-cacheable) loads; they are ordered
// after the producers' writes by thread 0's acquire fence in the grid barrier
// followed by the CTA barrier.  Phased engine: every vector is read-only for
// the kernel's lifetime and may use the read-only path.
template <bool INKERNEL>
__device__ __forceinline__ double ldx(const double *p)
{
    if (INKERNEL) return *p;
    return ld_keep_f64(p, policy_evict_last());
}
// The local pass's partial row sums: stored L2-resident (evict last) for the
// remote pass, which reads them once more (evict first: the line is about to
// be overwritten with the finished row).
__device__ __forceinline__ void st_partial_f64(double *p, double v)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v),
                 "l"(policy_evict_last())
                 : "memory");
}
__device__ __forceinline__ double ld_partial_f64(const double *p)
{
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;"
                 : "=d"(v)
                 : "l"(p), "l"(policy_evict_first())
                 : "memory");
    return v;
}
__device__ __forceinline__ float ld_keep_f32(const float *p, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
template <bool INKERNEL>
__device__ __forceinline__ float ldx(const float *p)
{
    if (INKERNEL) return *p;
    return ld_keep_f32(p, policy_evict_last());
}

// binary32 -> binary64, exact, from the two formats' field layouts (IEEE 754:
// sign | 8-bit exponent biased by 127 | 23 fraction bits, and sign | 11-bit
// exponent biased by 1023 | 52 fraction bits).  A normal number keeps its sign,
// its exponent gains 1023 - 127 = 896 and its fraction moves up 29 bits: a few
// integer operations instead of a conversion instruction, which GB300 runs at
// its (low) FP64 rate.  Zero keeps its sign; subnormals, infinities and NaNs
// take the conversion instruction.
__device__ __noinline__ double f2d_rare(float f)
{
    return (double)f;  // a call, so that the common path does not execute it predicated
}
__device__ __forceinline__ double f2d_exact(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t m = u & 0x7fffffffu;
    if (m - 0x00800000u < 0x7f000000u)  // exponent field 1..254
        return __hiloint2double((int)((u & 0x80000000u) | ((m >> 3) + 0x38000000u)),
                                (int)(m << 29));
    if (m == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
    return f2d_rare(f);
}

// binary64 -> binary32, rounded to nearest with ties to even (IEEE 754), for a
// result that is a normal binary32 number: the exponent loses 896, the 52-bit
// fraction keeps its top 23 bits, and the 29 dropped bits decide the rounding
// (above half, or exactly half with an odd last kept bit, adds one; a carry out
// of the fraction moves into the exponent, and past the largest finite value
// gives infinity, as the rounding rule requires).  Integer operations only;
// zero, results below the binary32 normal range, overflow, infinities and NaNs
// take the conversion instruction.
__device__ __noinline__ float d2f_rare(double d)
{
    return __double2float_rn(d);  // a call, so that the common path does not execute it predicated
}
__device__ __forceinline__ float d2f_rn(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned e = (unsigned)(u >> 52) & 0x7ffu;
    if (e - 897u <= 253u) {  // exponent field 897..1150: binary32 exponent 1..254
        const unsigned hi = (unsigned)(u >> 29) & 0x7fffffu;
        const unsigned rest = (unsigned)u & 0x1fffffffu;
        unsigned f = ((e - 896u) << 23) | hi;
        f += (rest > 0x10000000u || (rest == 0x10000000u && (hi & 1u))) ? 1u : 0u;
        return __uint_as_float(f | ((unsigned)(u >> 32) & 0x80000000u));
    }
    return d2f_rare(d);
}

// Value loads of the message steps: each value is read once per apply, so no
// L2 priority is asked for (an evict-last mark on every message buffer crowds
// out x, which the SpMV gathers keep resident).  Fused engine: plain loads.
template <bool INKERNEL, class T>
__device__ __forceinline__ T ldm(const T *p)
{
    if (INKERNEL) return *p;
    return __ldg(p);
}

// Batched element loop over [b, e): U independent index loads, then U
// independent data loads, then U stores, per thread and step.
// WAIT: the index arrays are constant plan data, so the index loads are issued
// before the programmatic-launch wait and only the value loads follow it.
template <int U, class T = double, bool WAIT = false, class LoadIdx, class LoadVal, class Store>
__device__ __forceinline__ void batched(int b, int e, int tid, LoadIdx li, LoadVal lv, Store st)
{
    for (int base = b + tid; base < e; base += NT * U) {
        uint32_t ix[U];
        T vv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) ix[u] = li(k);
        }
        if (WAIT) griddep_wait();
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) vv[u] = lv(k, ix[u]);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) st(k, ix[u], vv[u]);
        }
    }
}

// ------------------------------------------------------- three-block SpMV
struct Csr3 {
    const int32_t *rowptr;
    const uint32_t *colenc;
    const double *val;
    const float *val32;
};

template <bool INKERNEL, class XT>
__device__ __forceinline__ XT load_x(uint32_t c, const XT *x, const XT *bll, const XT *bnl)
{
    const uint32_t blk = c >> kBlockShift;
    const XT *src = blk == 0 ? x : (blk == 1 ? bll : bnl);
    return ldx<INKERNEL>(src + (c & kIndexMask));
}

// One stored entry into a row's sum.  FP64: one FMA.  FP32 values: the FP32
// product of the value and x rounded to FP32 (already FP32 when the sources
// hold FP32 copies), added in FP64.
template <class XT>
__device__ __forceinline__ double f32_product(float a, XT xv)
{
    float xf;
    if constexpr (sizeof(XT) == 4) xf = xv;
    else xf = d2f_rn(xv);
    return f2d_exact(__fmul_rn(a, xf));
}
template <bool F32, class XT>
__device__ __forceinline__ double entry_add(double acc, const double *val, const float *val32,
                                            int k, XT xv)
{
    if constexpr (F32) {
        return __dadd_rn(acc, f32_product(val32[k], xv));
    } else {
        static_assert(sizeof(XT) == 8, "FP64 values take FP64 sources");
        return fma(val[k], xv, acc);
    }
}

// Scaling of a row result: exact exponent arithmetic when scale is a power
// of two and the result stays normal (no FP64 instruction), else one DMUL.
struct Scale {
    double s;
    int e2;  // scale = 2^e2, or kNoPow2
};
constexpr int kNoPow2 = 1 << 30;
__device__ __forceinline__ double apply_scale(double acc, const Scale sc)
{
    if (sc.e2 == 0) return acc;  // scale 1 = 2^0 (an integer test: no FP64 compare per row)
    if (sc.e2 != kNoPow2) {
        const long long bits = __double_as_longlong(acc);
        const int ex = (int)((bits >> 52) & 0x7ff);
        if (ex > 0 && ex < 0x7ff && ex + sc.e2 > 0 && ex + sc.e2 < 0x7ff)
            return __longlong_as_double(bits + ((long long)sc.e2 << 52));
    }
    return __dmul_rn(sc.s, acc);
}

// ------------------------------------------- TMA-staged three-block SpMV
// A row tile's slices of the row pointer, column and value arrays are brought
// into shared memory by bulk asynchronous copies (cp.async.bulk, completion
// counted on an mbarrier), two stages per CTA, so the copy of the next tile
// overlaps the current one.  Slices are widened to 16-byte boundaries (the
// arrays are padded for that).  Each row is then summed by V lanes straight
// from shared memory, gathering x from HBM / L2: one DFMA per stored entry.

struct StageLayout {  // byte offsets inside one stage
    int rows, col, val, bytes;
};
__host__ __device__ __forceinline__ int align16(int b) { return (b + 15) & ~15; }
// vb: bytes per stored value (8 FP64, 4 FP32)
__host__ __device__ __forceinline__ StageLayout stage_layout(int cap, int tile_rows, int vb = 8)
{
    StageLayout L;
    L.rows = 0;
    L.col = align16(4 * (tile_rows + 8));
    L.val = L.col + align16(4 * (cap + 8));
    L.bytes = L.val + align16(vb * (cap + 8));
    return L;
}
constexpr int kMaxStages = 4;
constexpr int kMbarBytes = 16 * kMaxStages;  // one 8-byte mbarrier per stage, 16-byte slots

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    const uint64_t pol = policy_evict_first();  // the matrix is streamed once per apply
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], "
        "%2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, "
        "1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

struct TileStage {
    uint64_t *bar;
    int *rows;
    uint32_t *col;
    double *val;  // FP32 mode stores floats here
};

__device__ __forceinline__ TileStage tile_stage(unsigned char *base, int s, int cap, int tile_rows,
                                               int vb = 8)
{
    const StageLayout L = stage_layout(cap, tile_rows, vb);
    unsigned char *p = base + kMbarBytes + s * L.bytes;
    TileStage t;
    t.bar = reinterpret_cast<uint64_t *>(base + 16 * s);
    t.rows = reinterpret_cast<int *>(p + L.rows);
    t.col = reinterpret_cast<uint32_t *>(p + L.col);
    t.val = reinterpret_cast<double *>(p + L.val);
    return t;
}

// One thread: start the copies of the tile's slices into stage `st`.
template <bool F32>
__device__ __forceinline__ void tile_issue(const Csr3 &A, const TileStage &st, int r0, int r1,
                                           int k0, int k1)
{
    const int rb = r0 & ~3, re = (r1 + 1 + 3) & ~3;
    const int kb = k0 & ~3, ke = (k1 + 3) & ~3;
    const uint32_t brow = 4u * (re - rb), bcol = 4u * (ke - kb), bval = (F32 ? 4u : 8u) * (ke - kb);
    fence_proxy_async();  // earlier generic reads of this stage are ordered before the copies
    mbar_expect_tx(st.bar, brow + bcol + bval);
    bulk_g2s(st.rows, A.rowptr + rb, brow, st.bar);
    if (bcol) {
        bulk_g2s(st.col, A.colenc + kb, bcol, st.bar);
        if (F32)
            bulk_g2s(st.val, A.val32 + kb, bval, st.bar);
        else
            bulk_g2s(st.val, A.val + kb, bval, st.bar);
    }
}

// All threads: wait for the stage's copies (bounded).  On a timeout the error
// flag is set, the wait continues (bounded again) so that no copy is left in
// flight, and false is returned.
__device__ __forceinline__ bool tile_wait(const TileStage &st, uint32_t parity, int *err)
{
    constexpr long long kLimitNs = 2000000000ll;  // 2 s; a healthy copy takes microseconds
    if (mbar_try_wait(st.bar, parity)) return true;
    long long t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 256; i++)
            if (mbar_try_wait(st.bar, parity)) return true;
        if (globaltimer() - t0 > kLimitNs) break;
    }
    atomicCAS(err, 0, 2);
    t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 256; i++)
            if (mbar_try_wait(st.bar, parity)) return false;
        if (globaltimer() - t0 > kLimitNs) return false;
    }
}

// What a row sum covers: the whole three-block row (FULL), only its
// on_process part (LOCAL: the partial, unscaled, goes to y), or its remote
// part (REMOTE: the FMA chain continues from the partial in y, then scales).
enum SpmvMode { kFull = 0, kLocal = 1, kRemote = 2 };

// Rows [r0, r1) from a staged tile.  XT: element type of the three sources
// (FP32 copies in the phased engines' FP32 mode).  y32, when not null, receives
// each finished row rounded to FP32 (the next chained apply's source).
template <int V, bool F32, bool INKERNEL, int MODE = kFull, class XT = double>
__device__ __forceinline__ void tile_compute(const TileStage &st, const XT *x, const XT *bll,
                                             const XT *bnl, double *y, float *y32, const Scale sc,
                                             int r0, int r1, int k0, int tid)
{
    const int rb = r0 & ~3, kb = k0 & ~3;
    const int nr = r1 - r0;
    const int lane = tid & (V - 1), grp = tid / V, groups = NT / V;
    const float *val32 = reinterpret_cast<const float *>(st.val);
    for (int base = 0; base < nr; base += groups) {
        const int i = base + grp;
        double acc = 0.0;
        if (MODE == kRemote && i < nr && lane == 0) acc = ld_partial_f64(y + r0 + i);
        if (i < nr) {
            const int s = st.rows[r0 - rb + i] - kb, e = st.rows[r0 - rb + i + 1] - kb;
#pragma unroll 4
            for (int k = s + lane; k < e; k += V)
                acc = entry_add<F32>(acc, st.val, val32, k, load_x<INKERNEL>(st.col[k], x, bll, bnl));
        }
        if (V > 1) {
#pragma unroll
            for (int o = V / 2; o > 0; o >>= 1)
                acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        }
        if (i < nr && lane == 0) {
            if (MODE == kLocal) {
                st_partial_f64(y + r0 + i, acc);
            } else {
                const double r = apply_scale(acc, sc);
                y[r0 + i] = r;
                if (y32) y32[r0 + i] = d2f_rn(r);
            }
        }
    }
}

// A single row with more stored entries than a stage holds: read straight from
// global memory, the whole CTA on the row (fixed strides, fixed-order tree).
template <bool F32, bool INKERNEL, int MODE = kFull, class XT = double>
__device__ void row_direct(const Csr3 &A, const XT *x, const XT *bll, const XT *bnl, double *y,
                           float *y32, const Scale sc, int r0, int r1, double *red, int tid)
{
    for (int i = r0; i < r1; i++) {
        const int s = ld_stream_s32(A.rowptr + i), e = ld_stream_s32(A.rowptr + i + 1);
        double acc = 0.0;
        for (int k = s + tid; k < e; k += NT) {
            const XT xv = load_x<INKERNEL>(ld_stream_u32(A.colenc + k), x, bll, bnl);
            if constexpr (F32)
                acc = __dadd_rn(acc, f32_product(ld_stream_f32(A.val32 + k), xv));
            else
                acc = fma(ld_stream_f64(A.val + k), xv, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = MODE == kRemote ? y[i] : 0.0;
            for (int q = 0; q < NT / 32; q++) t = __dadd_rn(t, red[q]);
            if (MODE == kLocal) {
                y[i] = t;
            } else {
                const double r = apply_scale(t, sc);
                y[i] = r;
                if (y32) y32[i] = d2f_rn(r);
            }
        }
        __syncthreads();
    }
}

// Shared memory of the apply kernels: the mbarriers, `ns` stages, and a small
// reduction area for row_direct.
__host__ __device__ __forceinline__ int tile_smem_bytes(int cap, int tile_rows, int ns, int vb = 8)
{
    return kMbarBytes + ns * stage_layout(cap, tile_rows, vb).bytes + 8 * (NT / 32);
}
__device__ __forceinline__ double *tile_red(unsigned char *base, int cap, int tile_rows, int ns,
                                            int vb = 8)
{
    return reinterpret_cast<double *>(base + kMbarBytes +
                                      ns * stage_layout(cap, tile_rows, vb).bytes);
}
__device__ __forceinline__ void tile_smem_init(unsigned char *base, int ns)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; s++) mbar_init(reinterpret_cast<uint64_t *>(base + 16 * s), 1);
        fence_barrier_init();
    }
    __syncthreads();
}

// ------------------------------------------------- device-side waits
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Spin (bounded) until *p >= target; relaxed loads, the caller fences.
__device__ __forceinline__ bool wait_ge(const unsigned long long *p, unsigned long long target,
                                        int *err, long long timeout_ns)
{
    if (target == 0 || ld_relaxed(p) >= target) return true;
    const long long t0 = globaltimer();
    unsigned ns = 32;
    for (;;) {
        if (*(volatile int *)err) return false;
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        if (ld_relaxed(p) >= target) return true;
        if (globaltimer() - t0 > timeout_ns) {
            atomicCAS(err, 0, 1);
            return false;
        }
    }
}

// The element work of the message steps (shared by both engines; T = double,
// or float for the FP32 copies of the phased engines' FP32 mode).
template <bool INKERNEL, int U, class T = double, bool WAIT = false>
__device__ __noinline__ void step_gather(T *dst, const T *src, const int32_t *idx, int b, int e,
                                         int tid)
{
    const uint64_t pol = policy_evict_first();
    batched<U, T, WAIT>(
        b, e, tid, [&](int k) { return (uint32_t)ld_stream_hint_s32(idx + k, pol); },
        [&](int, uint32_t j) { return ldm<INKERNEL>(src + j); },
        [&](int k, uint32_t, T v) { dst[k] = v; });
}
template <bool INKERNEL, int U, class T = double, bool WAIT = false>
__device__ __noinline__ void step_pack(T *gsend, const T *x, const T *lbuf, const uint32_t *src,
                                       int b, int e, int tid)
{
    const uint64_t pol = policy_evict_first();
    batched<U, T, WAIT>(
        b, e, tid, [&](int k) { return ld_stream_hint_u32(src + k, pol); },
        [&](int, uint32_t u) {
            return (u & kFromLbuf) ? ldm<INKERNEL>(lbuf + (u & ~kFromLbuf)) : ldm<INKERNEL>(x + u);
        },
        [&](int k, uint32_t, T v) { gsend[k] = v; });
}
template <bool INKERNEL, int U, class T = double, bool WAIT = false>
__device__ __noinline__ void step_transfer(T *grecv, const T *gsend, const int32_t *dst, int b,
                                           int e, int tid)
{
    const uint64_t pol = policy_evict_first();
    batched<U, T, WAIT>(
        b, e, tid, [&](int k) { return (uint32_t)ld_stream_hint_s32(dst + k, pol); },
        [&](int k, uint32_t) { return ldm<INKERNEL>(gsend + k); },
        [&](int, uint32_t d, T v) { grecv[d] = v; });
}

__device__ __forceinline__ bool staged_tile(const Item &it, int cap)
{
    return it.kind == kSpmv && it.k1 - it.k0 <= cap;
}

// --------------------------------------------------------- phased engine
template <class T>
__global__ void __launch_bounds__(NT)
    k_gather2(const T *x, const int32_t *bll_j, T *bll, int n_bll, const int32_t *lbuf_j, T *lbuf,
              int n_lbuf, const int *err)
{
    // sticky error: no work until cleared (a flag set by the programmatic
    // predecessor itself is seen by the next launch)
    if (*(volatile const int *)err) return;
    const int per = NT * 8;
    for (int b = blockIdx.x * per; b < n_bll + n_lbuf; b += gridDim.x * per) {
        const int e = min(b + per, n_bll + n_lbuf);
        if (b < n_bll)
            step_gather<false, 8, T, true>(bll, x, bll_j, b, min(e, n_bll), threadIdx.x);
        if (e > n_bll) {
            const int lb = max(b, n_bll) - n_bll, le = e - n_bll;
            step_gather<false, 8, T, true>(lbuf, x, lbuf_j, lb, le, threadIdx.x);
        }
    }
    griddep_done();
}
template <class T>
__global__ void __launch_bounds__(NT)
    k_pack(const T *x, const T *lbuf, const uint32_t *src, T *gsend, int n, const int *err)
{
    if (*(volatile const int *)err) return;
    const int per = NT * 8;
    for (int b = blockIdx.x * per; b < n; b += gridDim.x * per)
        step_pack<false, 8, T, true>(gsend, x, lbuf, src, b, min(b + per, n), threadIdx.x);
    griddep_done();
}
template <class T>
__global__ void __launch_bounds__(NT)
    k_transfer(const T *gsend, const int32_t *dst, T *grecv, int n, const int *err)
{
    if (*(volatile const int *)err) return;
    const int per = NT * 8;
    for (int b = blockIdx.x * per; b < n; b += gridDim.x * per)
        step_transfer<false, 8, T, true>(grecv, gsend, dst, b, min(b + per, n), threadIdx.x);
    griddep_done();
}
template <class T>
__global__ void __launch_bounds__(NT)
    k_unpack(const T *grecv, const int32_t *src, T *bnl, int n, const int *err)
{
    if (*(volatile const int *)err) return;
    const int per = NT * 8;
    for (int b = blockIdx.x * per; b < n; b += gridDim.x * per)
        step_gather<false, 8, T, true>(bnl, grecv, src, b, min(b + per, n), threadIdx.x);
    griddep_done();
}
// FP32 copy of an input vector (first apply of a chain in FP32 mode)
__global__ void __launch_bounds__(NT) k_to_f32(const double *v, float *v32, int64_t n, const int *err)
{
    griddep_wait();
    if (*(volatile const int *)err) return;
    for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
        v32[i] = d2f_rn(ld_stream_f64(v + i));
    griddep_done();
}
template <int V, bool F32, int MODE = kFull>
__global__ void __launch_bounds__(NT)
    k_spmv(Csr3 A, const void *xs, const void *blls, const void *bnls, double *y, float *y32,
           Scale sc, const Item *tiles, int n_tiles, int cap, int trows, int ns, int *err)
{
    // FP32 mode: the three sources are FP32 copies
    using XT = typename std::conditional<F32, float, double>::type;
    const XT *x = static_cast<const XT *>(xs), *bll = static_cast<const XT *>(blls),
             *bnl = static_cast<const XT *>(bnls);
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    griddep_wait();
    if (*(volatile const int *)err) return;  // sticky error: no work until cleared
    constexpr int VB = F32 ? 4 : 8;
    tile_smem_init(smem, ns);
    double *red = tile_red(smem, cap, trows, ns, VB);
    uint32_t phase = 0;
    // a contiguous block of tiles per CTA (neighbouring rows share x and the
    // receive buffers of their process, which then stay in this SM's L1);
    // tile i of the block uses stage i % ns and is requested ns - 1 tiles ahead
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    const int q0 = blockIdx.x * per, q1 = min(n_tiles, q0 + per);
    if (tid == 0)
        for (int i = 0; i < ns - 1; i++) {
            const int q = q0 + i;
            if (q >= q1) break;
            const Item it = tiles[q];
            if (staged_tile(it, cap))
                tile_issue<F32>(A, tile_stage(smem, i, cap, trows, VB), it.b, it.e, it.k0, it.k1);
        }
    int cur = 0;
    for (int i = 0, q = q0; q < q1; i++, q++) {
        const Item it = tiles[q];
        const int qa = q + (ns - 1);
        if (tid == 0 && qa < q1) {
            const Item ita = tiles[qa];
            const int sa = (cur + ns - 1) % ns;  // the stage tile i - 1 used
            if (staged_tile(ita, cap))
                tile_issue<F32>(A, tile_stage(smem, sa, cap, trows, VB), ita.b, ita.e, ita.k0,
                                ita.k1);
        }
        if (staged_tile(it, cap)) {
            const TileStage st = tile_stage(smem, cur, cap, trows, VB);
            const bool ok = tile_wait(st, (phase >> cur) & 1, err);
            phase ^= 1u << cur;
            if (ok)
                tile_compute<V, F32, false, MODE>(st, x, bll, bnl, y, y32, sc, it.b, it.e, it.k0,
                                                  tid);
        } else {
            row_direct<F32, false, MODE>(A, x, bll, bnl, y, y32, sc, it.b, it.e, red, tid);
        }
        cur = cur + 1 == ns ? 0 : cur + 1;
        __syncthreads();
    }
    griddep_done();
}

// ------------------------------------------- remote pass with staged halos
// The overlapped engine's remote part with each process's receive buffers
// (its b_{l->l} and b_{nl->l} segments, contiguous in the workspace) staged in
// shared memory.  A CTA's run of tiles is cut at process boundaries
// (Item::msg = process); when the run enters a new process, one thread copies
// that process's two segments, widened to 16-byte boundaries, into the window
// with two bulk copies on their own mbarrier, and every remote gather of the
// process's rows then reads shared memory: each received value is read from
// global memory once per process, in order, instead of once per use.
__host__ __device__ __forceinline__ int halo_align(int elem_bytes) { return 16 / elem_bytes; }

template <int V, bool F32>
__device__ __forceinline__ void tile_compute_halo(const TileStage &st, const void *win, int bll_lo,
                                                  int nbw, int bnl_lo, double *y, float *y32,
                                                  const Scale sc, int r0, int r1, int k0, int tid)
{
    using XT = typename std::conditional<F32, float, double>::type;
    const XT *w = static_cast<const XT *>(win);
    const int rb = r0 & ~3, kb = k0 & ~3;
    const int nr = r1 - r0;
    const int lane = tid & (V - 1), grp = tid / V, groups = NT / V;
    const float *val32 = reinterpret_cast<const float *>(st.val);
    for (int base = 0; base < nr; base += groups) {
        const int i = base + grp;
        double acc = 0.0;
        if (i < nr && lane == 0) acc = ld_partial_f64(y + r0 + i);
        if (i < nr) {
            const int s = st.rows[r0 - rb + i] - kb, e = st.rows[r0 - rb + i + 1] - kb;
#pragma unroll 4
            for (int k = s + lane; k < e; k += V) {
                const uint32_t c = st.col[k];
                const int idx = (int)(c & kIndexMask);
                const XT xv = (c >> kBlockShift) == 1 ? w[idx - bll_lo] : w[nbw + idx - bnl_lo];
                acc = entry_add<F32>(acc, st.val, val32, k, xv);
            }
        }
        if (V > 1) {
#pragma unroll
            for (int o = V / 2; o > 0; o >>= 1)
                acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        }
        if (i < nr && lane == 0) {
            const double r = apply_scale(acc, sc);
            y[r0 + i] = r;
            if (y32) y32[r0 + i] = d2f_rn(r);
        }
    }
}

template <int V, bool F32>
__global__ void __launch_bounds__(NT)
    k_spmv_halo(Csr3 A, const void *blls, const void *bnls, double *y, float *y32, Scale sc,
                const Item *tiles, int n_tiles, int cap, int trows, int ns,
                const int32_t *bll_rank, const int32_t *bnl_rank, int *err)
{
    using XT = typename std::conditional<F32, float, double>::type;
    constexpr int VB = F32 ? 4 : 8;
    const int AL = halo_align((int)sizeof(XT));
    const XT *bll = static_cast<const XT *>(blls), *bnl = static_cast<const XT *>(bnls);
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    griddep_wait();
    if (*(volatile const int *)err) return;  // sticky error: no work until cleared
    const int base_bytes = tile_smem_bytes(cap, trows, ns, VB);
    uint64_t *wbar = reinterpret_cast<uint64_t *>(smem + base_bytes);
    XT *win = reinterpret_cast<XT *>(smem + base_bytes + 16);
    if (tid == 0) mbar_init(wbar, 1);
    tile_smem_init(smem, ns);  // the stage barriers, fence and CTA barrier
    double *red = tile_red(smem, cap, trows, ns, VB);
    TileStage wst{};
    wst.bar = wbar;
    uint32_t phase = 0, wphase = 0;
    int cur_rank = -1, bll_lo = 0, nbw = 0, bnl_lo = 0;
    bool wok = false;
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    const int q0 = blockIdx.x * per, q1 = min(n_tiles, q0 + per);
    if (tid == 0)
        for (int i = 0; i < ns - 1; i++) {
            const int q = q0 + i;
            if (q >= q1) break;
            const Item it = tiles[q];
            if (staged_tile(it, cap))
                tile_issue<F32>(A, tile_stage(smem, i, cap, trows, VB), it.b, it.e, it.k0, it.k1);
        }
    int cur = 0;
    for (int q = q0; q < q1; q++) {
        const Item it = tiles[q];
        const int qa = q + (ns - 1);
        if (tid == 0 && qa < q1) {
            const Item ita = tiles[qa];
            const int sa = (cur + ns - 1) % ns;
            if (staged_tile(ita, cap))
                tile_issue<F32>(A, tile_stage(smem, sa, cap, trows, VB), ita.b, ita.e, ita.k0,
                                ita.k1);
        }
        if (it.msg != cur_rank) {
            // every thread finished the previous tile (CTA barrier at the end of
            // the last iteration): the window may be refilled
            const int t = it.msg;
            const int b0 = bll_rank[t] & ~(AL - 1), b1 = (bll_rank[t + 1] + AL - 1) & ~(AL - 1);
            const int n0 = bnl_rank[t] & ~(AL - 1), n1 = (bnl_rank[t + 1] + AL - 1) & ~(AL - 1);
            if (tid == 0) {
                fence_proxy_async();
                mbar_expect_tx(wbar, (uint32_t)((b1 - b0) + (n1 - n0)) * (uint32_t)sizeof(XT));
                if (b1 > b0) bulk_g2s(win, bll + b0, (uint32_t)(b1 - b0) * sizeof(XT), wbar);
                if (n1 > n0)
                    bulk_g2s(win + (b1 - b0), bnl + n0, (uint32_t)(n1 - n0) * sizeof(XT), wbar);
            }
            bll_lo = b0;
            nbw = b1 - b0;
            bnl_lo = n0;
            wok = tile_wait(wst, wphase, err);
            wphase ^= 1;
            cur_rank = t;
        }
        if (staged_tile(it, cap)) {
            const TileStage st = tile_stage(smem, cur, cap, trows, VB);
            const bool ok = tile_wait(st, (phase >> cur) & 1, err);
            phase ^= 1u << cur;
            if (ok && wok)
                tile_compute_halo<V, F32>(st, win, bll_lo, nbw, bnl_lo, y, y32, sc, it.b, it.e,
                                          it.k0, tid);
        } else if (wok) {
            // a row longer than a stage: entries from global memory, values
            // from the window (the whole CTA on the row, fixed-order tree)
            for (int r = it.b; r < it.e; r++) {
                const int s0 = ld_stream_s32(A.rowptr + r), e0 = ld_stream_s32(A.rowptr + r + 1);
                double acc = 0.0;
                for (int k = s0 + tid; k < e0; k += NT) {
                    const uint32_t c = ld_stream_u32(A.colenc + k);
                    const int idx = (int)(c & kIndexMask);
                    const XT xv = (c >> kBlockShift) == 1 ? win[idx - bll_lo]
                                                          : win[nbw + idx - bnl_lo];
                    if constexpr (F32)
                        acc = __dadd_rn(acc, f32_product(ld_stream_f32(A.val32 + k), xv));
                    else
                        acc = fma(ld_stream_f64(A.val + k), xv, acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
                if ((tid & 31) == 0) red[tid >> 5] = acc;
                __syncthreads();
                if (tid == 0) {
                    double t2 = ld_partial_f64(y + r);
                    for (int w2 = 0; w2 < NT / 32; w2++) t2 = __dadd_rn(t2, red[w2]);
                    const double res = apply_scale(t2, sc);
                    y[r] = res;
                    if (y32) y32[r] = d2f_rn(res);
                }
                __syncthreads();
            }
        }
        cur = cur + 1 == ns ? 0 : cur + 1;
        __syncthreads();
    }
    griddep_done();
}

// ----------------------------------------------- warp-pipelined SpMV
// Each warp owns `ns` shared-memory stages with their own mbarriers and
// streams its own tiles (at most 32 / V rows and `capw` entries): lane 0
// issues the bulk copies of the tile ns - 1 ahead, the warp waits on its
// stage, sums its rows, and only synchronises with itself before the stage is
// reused.  No CTA-wide barrier: a warp whose gathers hit is not held back by
// one whose gathers miss.
constexpr int WPB = NT / 32;  // warps per CTA

__host__ __device__ __forceinline__ int warp_smem_bytes(int capw, int rowsw, int ns, int vb = 8)
{
    return 16 * kMaxStages * WPB + WPB * ns * stage_layout(capw, rowsw, vb).bytes;
}

// One row summed by a whole warp straight from global memory (lanes stride the
// row, fixed xor tree); REMOTE adds the partial to the warp's sum.
template <bool F32, int MODE, bool INKERNEL = false, class XT>
__device__ __forceinline__ void row_warp(const Csr3 &A, const XT *x, const XT *bll, const XT *bnl,
                                         double *y, float *y32, const Scale sc, int r, int lane)
{
    const int s0 = ld_stream_s32(A.rowptr + r), e0 = ld_stream_s32(A.rowptr + r + 1);
    double acc = 0.0;
    for (int k = s0 + lane; k < e0; k += 32) {
        const XT xv = load_x<INKERNEL>(ld_stream_u32(A.colenc + k), x, bll, bnl);
        if constexpr (F32)
            acc = __dadd_rn(acc, f32_product(ld_stream_f32(A.val32 + k), xv));
        else
            acc = fma(ld_stream_f64(A.val + k), xv, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) {
        if (MODE == kRemote) acc = __dadd_rn(y[r], acc);
        if (MODE == kLocal) {
            y[r] = acc;
        } else {
            const double res = apply_scale(acc, sc);
            y[r] = res;
            if (y32) y32[r] = d2f_rn(res);
        }
    }
}

template <int V, bool F32, int MODE>
__global__ void __launch_bounds__(NT, 4)
    k_spmv_w(Csr3 A, const void *xs, const void *blls, const void *bnls, double *y, float *y32,
             Scale sc, const Item *tiles, int n_tiles, int capw, int rowsw, int ns, int *err)
{
    using XT = typename std::conditional<F32, float, double>::type;
    const XT *x = static_cast<const XT *>(xs), *bll = static_cast<const XT *>(blls),
             *bnl = static_cast<const XT *>(bnls);
    extern __shared__ __align__(16) unsigned char smem[];
    griddep_wait();
    if (*(volatile const int *)err) return;  // sticky error: no work until cleared
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const StageLayout L = stage_layout(capw, rowsw, F32 ? 4 : 8);
    unsigned char *mine = smem + 16 * kMaxStages * WPB + warp * ns * L.bytes;
    auto stage = [&](int s2) {
        TileStage t;
        t.bar = reinterpret_cast<uint64_t *>(smem + 16 * (warp * kMaxStages + s2));
        unsigned char *p = mine + s2 * L.bytes;
        t.rows = reinterpret_cast<int *>(p + L.rows);
        t.col = reinterpret_cast<uint32_t *>(p + L.col);
        t.val = reinterpret_cast<double *>(p + L.val);
        return t;
    };
    if (lane == 0) {
        for (int s2 = 0; s2 < ns; s2++) mbar_init(stage(s2).bar, 1);
        fence_barrier_init();
    }
    __syncwarp();
    // a contiguous block of tiles per CTA, its warps interleaved inside it
    const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
    const int q0 = blockIdx.x * per, q1 = min(n_tiles, q0 + per);
    if (lane == 0)
        for (int i = 0; i < ns - 1; i++) {
            const int q = q0 + warp + i * WPB;
            if (q >= q1) break;
            const Item it = tiles[q];
            if (staged_tile(it, capw)) tile_issue<F32>(A, stage(i), it.b, it.e, it.k0, it.k1);
        }
    uint32_t phase = 0;
    int cur = 0;
    for (int q = q0 + warp; q < q1; q += WPB) {
        const Item it = tiles[q];
        const int qa = q + (ns - 1) * WPB;
        if (lane == 0 && qa < q1) {
            const Item ita = tiles[qa];
            if (staged_tile(ita, capw))
                tile_issue<F32>(A, stage((cur + ns - 1) % ns), ita.b, ita.e, ita.k0, ita.k1);
        }
        const int nr = it.e - it.b;
        if (staged_tile(it, capw)) {
            const TileStage st = stage(cur);
            const bool ok = tile_wait(st, (phase >> cur) & 1, err);
            phase ^= 1u << cur;
            if (ok) {
                const int rb = it.b & ~3, kb = it.k0 & ~3;
                const int sub = lane & (V - 1), grp = lane / V;
                const float *val32 = reinterpret_cast<const float *>(st.val);
                for (int base = 0; base < nr; base += 32 / V) {
                    const int i = base + grp;
                    double acc = 0.0;
                    if (MODE == kRemote && i < nr && sub == 0) acc = ld_partial_f64(y + it.b + i);
                    if (i < nr) {
                        const int s0 = st.rows[it.b - rb + i] - kb, e0 = st.rows[it.b - rb + i + 1] - kb;
#pragma unroll 4
                        for (int k = s0 + sub; k < e0; k += V)
                            acc = entry_add<F32>(acc, st.val, val32, k,
                                                 load_x<false>(st.col[k], x, bll, bnl));
                    }
                    if (V > 1) {
#pragma unroll
                        for (int o = V / 2; o > 0; o >>= 1)
                            acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
                    }
                    if (i < nr && sub == 0) {
                        if (MODE == kLocal) {
                            st_partial_f64(y + it.b + i, acc);
                        } else {
                            const double r = apply_scale(acc, sc);
                            y[it.b + i] = r;
                            if (y32) y32[it.b + i] = d2f_rn(r);
                        }
                    }
                }
            }
        } else {
            // a row longer than a warp stage: the warp sums it from global memory
            for (int r = it.b; r < it.e; r++) row_warp<F32, MODE>(A, x, bll, bnl, y, y32, sc, r, lane);
        }
        cur = cur + 1 == ns ? 0 : cur + 1;
        __syncwarp();
    }
    griddep_done();
}

// --------------------------------------------------- sliced-row SpMV
// NAPSPMV_PIPELINE_SELL: one lane per row over chunks of up to 32 rows of
// similar length stored column-major (slot first + i * lanes + lane).  A warp
// reads a chunk's columns and values as consecutive slots, coalesced, straight
// from global memory (no shared-memory stage, so occupancy is bounded by
// registers only), and every lane of a DFMA carries an entry: the rows of a
// chunk have similar counts.  Each row is summed in its stored order, one DFMA
// per entry (FP32 mode: FP32 product, FP64 add): the bits of the one-lane CSR
// kernels.  Chunks go to CTAs in groups, one chunk per warp (see k_spmv_s).
// Rows longer than kSellLong entries are summed afterwards by whole warps from
// the CSR part.
struct SellView {
    const int2 *info;
    const int32_t *perm;
    const uint32_t *col;
    const double *val;
    const float *val32;
    const int32_t *lrows;
    Csr3 A;  // the same part as CSR (long rows)
    int32_t nch, n_long;
};

__device__ __forceinline__ double ld_stream_hint_f64(const double *p, uint64_t pol)
{
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_stream_hint_f32(const float *p, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

// One chunk of a sliced-row part: lane `lane` sums the row of its slot in
// the chunk (nothing if the chunk has fewer rows), U entries at a time: U
// column loads and U value loads (coalesced across the warp, streamed with an
// L2 evict-first mark), U gathers of x or the receive buffers, then U FMAs
// in stored order.  INKERNEL: the sources are written earlier in the same
// launch (the fused engine): coherent loads instead of the read-only path.
template <bool F32, bool INKERNEL, int MODE, int U, class XT>
__device__ __forceinline__ void sell_chunk(const SellView &S, int c, const XT *x, const XT *bll,
                                           const XT *bnl, double *y, float *y32, const Scale sc,
                                           int lane, uint64_t pol)
{
    using VT = typename std::conditional<F32, float, double>::type;
    const int2 inf = S.info[c];
    const int width = inf.y >> 6, nl = inf.y & 63;
    if (lane >= nl) return;
    const int row = S.perm[32 * c + lane];
    double acc = MODE == kRemote ? ld_partial_f64(y + row) : 0.0;
    const int64_t base = (int64_t)inf.x + lane;
    for (int i = 0; i < width; i += U) {
        uint32_t cc[U];
        VT a[U];
        XT xv[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            cc[u] = i + u < width ? ld_stream_hint_u32(S.col + base + (int64_t)(i + u) * nl, pol)
                                  : kSellPad;
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t q = base + (int64_t)(i + u) * nl;
            if constexpr (F32)
                a[u] = cc[u] != kSellPad ? ld_stream_hint_f32(S.val32 + q, pol) : 0.0f;
            else
                a[u] = cc[u] != kSellPad ? ld_stream_hint_f64(S.val + q, pol) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            xv[u] = cc[u] != kSellPad ? load_x<INKERNEL>(cc[u], x, bll, bnl) : XT(0);
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (cc[u] != kSellPad) {
                if constexpr (F32) acc = __dadd_rn(acc, f32_product(a[u], xv[u]));
                else acc = fma(a[u], xv[u], acc);
            }
        }
    }
    if (MODE == kLocal) {
        st_partial_f64(y + row, acc);
    } else {
        const double r = apply_scale(acc, sc);
        y[row] = r;
        if (y32) y32[row] = d2f_rn(r);
    }
}

// Chunks are handed out in groups of W consecutive chunks (one per warp of a
// CTA of W warps), group g to CTA g mod grid: every CTA sweeps the arrays
// together with the others, so the pages in use at any time stay few.
// Measured on the 2^23-row banded random workload (FP64): contiguous runs of
// chunks per CTA, which spread ~900 CTAs over 3.4 GB of matrix and receive
// buffers, took 1.42 ms; groups of 8 handed out this way, 0.70 ms.  Four
// entries per step suit short rows (the stencils), eight longer ones.
// kSellGroup: the group of the 8-warp CTAs (the fused engine's).
constexpr int kSellGroup = 8;

template <bool F32, int MODE, int U, int W = 8>
__global__ void __launch_bounds__(32 * W, W == 8 ? (U >= 8 ? 4 : 6) : 1)
    k_spmv_s(SellView S, const void *xs, const void *blls, const void *bnls, double *y, float *y32,
             Scale sc, int *err)
{
    using XT = typename std::conditional<F32, float, double>::type;
    constexpr int WPB = W, G = W;
    const XT *x = static_cast<const XT *>(xs), *bll = static_cast<const XT *>(blls),
             *bnl = static_cast<const XT *>(bnls);
    griddep_wait();
    if (*(volatile const int *)err) return;  // sticky error: no work until cleared
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t pol = policy_evict_first();  // the matrix streams once per apply
    const int ngroups = (S.nch + G - 1) / G;
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x)
        for (int c = g * G + warp; c < min(S.nch, (g + 1) * G); c += WPB)
            sell_chunk<F32, false, MODE, U>(S, c, x, bll, bnl, y, y32, sc, lane, pol);
    // rows longer than kSellLong: a warp each
    const int gw = blockIdx.x * WPB + warp, nw = gridDim.x * WPB;
    for (int q = gw; q < S.n_long; q += nw) row_warp<F32, MODE>(S.A, x, bll, bnl, y, y32, sc, S.lrows[q], lane);
    griddep_done();
}

// ---------------------------------------------------------- fused engine
// One persistent, cooperative launch for every chained apply of one or more
// independent jobs (a batch).  Each apply runs in five levels separated by
// grid-wide barriers:
//   level 0  the on_node -> on_node and on_node -> off_node gathers (Eqs. IL2,
//            IL0); with composed gathers, both receive buffers from x
//   level 1  packing of g_send (Eq. I) and the inter-node transfer g_send ->
//            g_recv: the thread that packs element k also moves element k (it
//            reads back the g_send value it wrote), so no barrier separates
//            the two steps
//   level 2  off_node -> on_node: unpack into b_{nl->l} (Eq. IL1)
//   level 3  the three-block SpMV over the sliced rows (each row on_process,
//            on_node, off_node in one FMA chain)
// Splitting the rows into a local part overlapping levels 0-2 and a remote
// part (the overlap Algorithm NAPSpMV allows) was measured slower on GB300:
// the remote part's continuation of every row costs more than the local part
// hides (3D 7-point 128^3: 152 against ~100 us per apply).  Within a level the
// units of all jobs (message chunks of `chunk` elements, groups of
// kSellGroup sliced-row chunks, groups of 8 long rows) are dealt to the CTAs
// round robin: no ticket counter, no per-item dependency check, one barrier
// per level.  Every CTA of the
// cooperative launch is resident, so the barrier cannot wait on a CTA that
// never runs; its wait is bounded all the same.
constexpr int kLevels = 4;
// Elements per thread per pass in the message levels, and sliced-row entries
// per step in level 3, whatever the row lengths.  With these the kernel fits
// its 64 registers (4 CTAs per SM) without spilling.  Measured per apply on
// GB300 (3D 7-point 128^3 / Q1 2048^2 / 2^23-row banded random, FP64):
// 8 elements and 4 (8 for the long rows of the banded matrix) entries took
// 124 / 223 / 2,058 us; 4 elements 106 / 200 / 1,881 us; 2 elements with 4
// entries for every matrix 106 / 199 / 1,633 us.  Three elements per thread
// at 6 CTAs per SM (40 registers) spilled and ran slower on every workload.
constexpr int kFusedU = 2;
constexpr int kFusedSellU = 4;

struct FJob {
    SellView F;                   // the whole matrix, sliced rows
    const int32_t *src0, *src1;   // level-0 gathers: J2 / J0 (composed: BLL / BNL lists)
    int32_t n0, n1;
    const uint32_t *pack_src;
    const int32_t *xfer_dst, *unp_src;
    int32_t n_gs, n_bnl;
    int32_t composed, reps;
    Scale scale;
    double *bll, *lbuf, *gsend, *grecv, *bnl, *xtmp;
    int *err;
    const double *v;
    double *w;
    int32_t nmsg[kLevels];      // message units per level
    int32_t ch;                 // elements per message unit (option chunk)
    int32_t nunits[kLevels];    // all units per level
};

template <int MAXJ>
struct FusedParams {
    int32_t njobs, kmax, stall;
    long long timeout_ns, barrier_ns;
    unsigned int *bar;                 // [0] arrivals, [1] generation (zeroed before launch)
    unsigned long long *stallctr;      // a counter nothing increments (test hook)
    int32_t off[kLevels][MAXJ + 1];    // first unit of every job in each level
    FJob jobs[MAXJ];
};
static_assert(sizeof(FusedParams<64>) <= 32764, "kernel parameters are limited to 32,764 bytes");

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch: arrival count and generation.
// Thread 0 releases the CTA's writes (ordered by the CTA barrier) with its
// arrival, waits (bounded) for the generation to move, and acquires; the CTA
// barrier then orders every thread's later loads after it.  The last CTA to
// arrive resets the count before it publishes the next generation.  A wait
// that runs out sets every job's error flag and returns false: the CTA stops.
template <int MAXJ>
__device__ bool grid_barrier(const FusedParams<MAXJ> &prm)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *cnt = prm.bar, *gen = prm.bar + 1;
        const unsigned g = ld_acquire_u32(gen);
        fence_acq_rel();
        int ok = 1;
        if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
            atomicExch(cnt, 0u);
            fence_acq_rel();
            st_release_u32(gen, g + 1);
        } else {
            const long long t0 = globaltimer();
            unsigned ns = 32;
            while (ld_acquire_u32(gen) == g) {
                __nanosleep(ns);
                if (ns < 512) ns <<= 1;
                if (globaltimer() - t0 > prm.barrier_ns) {
                    for (int j = 0; j < prm.njobs; j++) atomicCAS(prm.jobs[j].err, 0, 1);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Pack and transfer of elements [b, e) in one pass: per element its pack
// source and destination index first, then the value, g_send written, the
// value read back from g_send and moved into g_recv.
__device__ __noinline__ void step_pack_transfer(double *gsend, double *grecv, const double *x,
                                                const double *lbuf, const uint32_t *src,
                                                const int32_t *dst, int b, int e, int tid)
{
    const uint64_t pol = policy_evict_first();
    constexpr int U = kFusedU;
    for (int base = b + tid; base < e; base += NT * U) {
        uint32_t sv[U];
        int32_t dv[U];
        double vv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) {
                sv[u] = ld_stream_hint_u32(src + k, pol);
                dv[u] = ld_stream_hint_s32(dst + k, pol);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) vv[u] = (sv[u] & kFromLbuf) ? lbuf[sv[u] & ~kFromLbuf] : x[sv[u]];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) gsend[k] = vv[u];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) vv[u] = *(volatile const double *)(gsend + k);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int k = base + u * NT;
            if (k < e) grecv[dv[u]] = vv[u];
        }
    }
}

// One unit of level `lvl` of job J (see the level list above).
template <bool F32>
__device__ __forceinline__ void fused_unit(const FJob &J, int lvl, int u, const double *x, double *y,
                                           int tid)
{
    const int warp = tid >> 5, lane = tid & 31;
    const uint64_t pol = policy_evict_first();
    if (u < J.nmsg[lvl]) {
        const int b = u * J.ch;
        switch (lvl) {
        case 0: {
            const int nu0 = (J.n0 + J.ch - 1) / J.ch;
            if (u < nu0) {
                step_gather<true, kFusedU>(J.bll, x, J.src0, b, min(J.n0, b + J.ch), tid);
            } else {
                const int b1 = (u - nu0) * J.ch;
                step_gather<true, kFusedU>(J.composed ? J.bnl : J.lbuf, x, J.src1, b1,
                                     min(J.n1, b1 + J.ch), tid);
            }
            break;
        }
        case 1:
            step_pack_transfer(J.gsend, J.grecv, x, J.lbuf, J.pack_src, J.xfer_dst, b,
                               min(J.n_gs, b + J.ch), tid);
            break;
        default:
            step_gather<true, kFusedU>(J.bnl, J.grecv, J.unp_src, b, min(J.n_bnl, b + J.ch), tid);
            break;
        }
        return;
    }
    // level 3: chunk groups of the sliced rows, then groups of 8 long rows
    u -= J.nmsg[lvl];
    const int ng = (J.F.nch + kSellGroup - 1) / kSellGroup;
    if (u < ng) {
        for (int c = u * kSellGroup + warp; c < min(J.F.nch, (u + 1) * kSellGroup); c += WPB)
            sell_chunk<F32, true, kFull, kFusedSellU>(J.F, c, x, J.bll, J.bnl, y, nullptr, J.scale,
                                                      lane, pol);
    } else {
        const int q = (u - ng) * WPB + warp;
        if (q < J.F.n_long)
            row_warp<F32, kFull, true>(J.F.A, x, J.bll, J.bnl, y, nullptr, J.scale, J.F.lrows[q], lane);
    }
}

template <bool F32, int MAXJ>
__global__ void __launch_bounds__(NT, 4) k_fused(const __grid_constant__ FusedParams<MAXJ> prm)
{
    const int tid = threadIdx.x;
    __shared__ int s_skip[MAXJ];
    for (int k = 0; k < prm.kmax; k++) {
        for (int lvl = 0; lvl < kLevels; lvl++) {
            // a job whose flag is set (a wait ran out, in this launch or before)
            // skips its work; nothing inside a level waits, so the flag is read
            // once per level (after the barrier that ended the previous one)
            const int g = (int)gridDim.x;
            if (tid < prm.njobs) {
                int skip = *(volatile int *)prm.jobs[tid].err;
                // test hook: the CTA holding job 0's first unit waits on a
                // counter nothing increments
                if (!skip && prm.stall && tid == 0 && k == 0 && lvl == 0 &&
                    (int)blockIdx.x == prm.off[0][0] % g &&
                    !wait_ge(prm.stallctr, 1, prm.jobs[0].err, prm.timeout_ns))
                    skip = 1;
                s_skip[tid] = skip;
            }
            __syncthreads();
            for (int j = 0; j < prm.njobs; j++) {
                const FJob &J = prm.jobs[j];
                if (k >= J.reps || s_skip[j]) continue;
                const double *x = (k == 0) ? J.v : (((J.reps - k) & 1) == 0 ? J.w : J.xtmp);
                double *y = (((J.reps - 1 - k) & 1) == 0) ? J.w : J.xtmp;
                const int base = prm.off[lvl][j];
                // units u with (base + u) mod grid == this CTA
                int u = (int)blockIdx.x - base % g;
                if (u < 0) u += g;
                for (; u < J.nunits[lvl]; u += g) fused_unit<F32>(J, lvl, u, x, y, tid);
            }
            if (!grid_barrier(prm)) return;
        }
    }
}

// ------------------------------------------------------------- dispatch
template <int MAXJ>
struct FusedKernelTable {
    using Fn = void (*)(const FusedParams<MAXJ>);
    static Fn get(bool f32) { return f32 ? k_fused<true, MAXJ> : k_fused<false, MAXJ>; }
};

static bool valid_vec(int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32; }

napspmv_opts resolve_opts(const napspmv_plan_t *P, const napspmv_opts *o)
{
    napspmv_opts r = P->defaults;
    if (!o) return r;
    r.precision = o->precision;  // 0 is FP64, a real choice
    if (o->engine) r.engine = o->engine;
    if (o->vec) r.vec = o->vec;
    if (o->ctas_per_sm) r.ctas_per_sm = o->ctas_per_sm;
    if (o->chunk) r.chunk = o->chunk;
    if (o->tile_rows) r.tile_rows = o->tile_rows;
    if (o->tile_nnz) r.tile_nnz = o->tile_nnz;
    if (o->stages) r.stages = o->stages;
    if (o->pipeline) r.pipeline = o->pipeline;
    if (o->halo) r.halo = o->halo;
    if (o->timeout_ms) r.timeout_ms = o->timeout_ms;
    r.debug_stall = o->debug_stall;
    return r;
}

static size_t smem_bytes(int32_t tile_nnz, int32_t tile_rows, int32_t ns = 2, int vb = 8)
{
    return (size_t)tile_smem_bytes(tile_nnz, tile_rows, ns, vb);
}

int build_items(napspmv_plan_t *P, int32_t tile_rows, int32_t tile_nnz)
{
    if (tile_rows < 1 || tile_nnz < 32 || smem_bytes(tile_nnz, tile_rows) > 200 * 1024) {
        set_error(NAPSPMV_ERR_ARG, "need tile_rows >= 1, tile_nnz >= 32 and two tile stages "
                                   "(12 B per entry, 4 B per row) within 200 KiB");
        return NAPSPMV_ERR_ARG;
    }
    ItemSet &S = P->items;
    if (S.d_items && S.tile_rows == tile_rows && S.tile_nnz == tile_nnz) return NAPSPMV_OK;
    const int nn = P->nn;
    // CTA tiles of the whole matrix, cut within each node's rows
    std::vector<Item> items;
    const std::vector<int32_t> &rp = P->h_rowptr;
    for (int x = 0; x < nn; x++) {
        int64_t r = P->node_rows[x];
        const int64_t end = P->node_rows[x + 1];
        while (r < end) {
            int64_t e = r;
            while (e < end && e - r < tile_rows && rp[e + 1] - rp[r] <= tile_nnz) e++;
            if (e == r) e = r + 1;  // one row longer than the capacity
            Item it{};
            it.kind = kSpmv;
            it.node = x;
            it.b = (int32_t)r;
            it.e = (int32_t)e;
            it.k0 = rp[r];
            it.k1 = rp[e];
            items.push_back(it);
            r = e;
        }
    }

    // tiles of the local / remote parts (overlapped engine), same size limits
    auto cut = [&](const std::vector<int32_t> &rp2, std::vector<Item> &out) {
        const int64_t n = (int64_t)rp2.size() - 1;
        int64_t r = 0;
        while (r < n) {
            int64_t e = r;
            while (e < n && e - r < tile_rows && rp2[e + 1] - rp2[r] <= tile_nnz) e++;
            if (e == r) e = r + 1;
            Item it{};
            it.kind = kSpmv;
            it.b = (int32_t)r;
            it.e = (int32_t)e;
            it.k0 = rp2[r];
            it.k1 = rp2[e];
            out.push_back(it);
            r = e;
        }
    };
    std::vector<Item> tl, tr, trh;
    if (!P->h_rowptrL.empty()) {
        cut(P->h_rowptrL, tl);
        cut(P->h_rowptrR, tr);
        if (!(P->flags & NAPSPMV_PARTITION_STRIDED)) {
            // remote tiles never straddle two processes: Item::msg is the
            // process, whose receive buffers the remote pass may stage
            const int64_t n = P->n, q = n / P->np, rem = n % P->np;
            std::vector<int32_t> sub;
            for (int32_t r = 0; r < P->np; r++) {
                const int64_t r0 = r * q + std::min<int64_t>(r, rem);
                const int64_t r1 = r0 + q + (r < rem ? 1 : 0);
                sub.assign(P->h_rowptrR.begin() + r0, P->h_rowptrR.begin() + r1 + 1);
                const size_t first = trh.size();
                cut(sub, trh);
                for (size_t k = first; k < trh.size(); k++) {
                    trh[k].b += (int32_t)r0;
                    trh[k].e += (int32_t)r0;
                    trh[k].msg = r;
                }
            }
        }
    }
    // warp tiles: the same cutting with a warp's share of a CTA tile
    std::vector<Item> wt, wtl, wtr;
    {
        const int32_t trows = tile_rows, tnnz = tile_nnz;
        tile_rows = std::max(1, trows / 8);
        tile_nnz = std::max(32, tnnz / 8);
        cut(P->h_rowptr, wt);
        if (!P->h_rowptrL.empty()) {
            cut(P->h_rowptrL, wtl);
            cut(P->h_rowptrR, wtr);
        }
        tile_rows = trows;
        tile_nnz = tnnz;
    }
    // the stage each list needs: its largest tile that is staged at all
    auto fit = [](const std::vector<Item> &v, int32_t tnnz, int32_t &cap, int32_t &rows) {
        cap = 32;
        rows = 1;
        for (const Item &it : v)
            if (it.kind == kSpmv && it.k1 - it.k0 <= tnnz) {
                cap = std::max(cap, it.k1 - it.k0);
                rows = std::max(rows, it.e - it.b);
            }
        cap = std::min(tnnz, (cap + 15) & ~15);
    };
    {
        const int32_t wn = std::max(32, tile_nnz / 8);
        fit(items, tile_nnz, S.fit_nnz[0], S.fit_rows[0]);
        fit(tl, tile_nnz, S.fit_nnz[1], S.fit_rows[1]);
        fit(tr, tile_nnz, S.fit_nnz[2], S.fit_rows[2]);
        fit(trh, tile_nnz, S.fit_nnz[6], S.fit_rows[6]);
        fit(wt, wn, S.fit_nnz[3], S.fit_rows[3]);
        fit(wtl, wn, S.fit_nnz[4], S.fit_rows[4]);
        fit(wtr, wn, S.fit_nnz[5], S.fit_rows[5]);
    }
    auto upload_items = [&](const std::vector<Item> &v, Item **d, int32_t *n) -> int {
        if (*d) cudaFree(*d);
        *d = nullptr;
        *n = (int32_t)v.size();
        if (v.empty()) return NAPSPMV_OK;
        NAP_CUDA(cudaMalloc(d, sizeof(Item) * v.size()));
        NAP_CUDA(cudaMemcpy(*d, v.data(), sizeof(Item) * v.size(), cudaMemcpyHostToDevice));
        return NAPSPMV_OK;
    };
    if (int rc = upload_items(wt, &S.d_wt, &S.n_wt)) return rc;
    if (int rc = upload_items(trh, &S.d_tilesRH, &S.n_tilesRH)) return rc;
    if (int rc = upload_items(wtl, &S.d_wtL, &S.n_wtL)) return rc;
    if (int rc = upload_items(wtr, &S.d_wtR, &S.n_wtR)) return rc;
    Item *d_tl = nullptr, *d_tr = nullptr;
    if (!tl.empty()) {
        NAP_CUDA(cudaMalloc(&d_tl, sizeof(Item) * tl.size()));
        NAP_CUDA(cudaMalloc(&d_tr, sizeof(Item) * tr.size()));
        NAP_CUDA(cudaMemcpy(d_tl, tl.data(), sizeof(Item) * tl.size(), cudaMemcpyHostToDevice));
        NAP_CUDA(cudaMemcpy(d_tr, tr.data(), sizeof(Item) * tr.size(), cudaMemcpyHostToDevice));
    }
    if (S.d_tilesL) cudaFree(S.d_tilesL);
    if (S.d_tilesR) cudaFree(S.d_tilesR);
    S.d_tilesL = d_tl;
    S.d_tilesR = d_tr;
    S.n_tilesL = (int32_t)tl.size();
    S.n_tilesR = (int32_t)tr.size();

    Item *d_items = nullptr;
    if (!items.empty()) {
        NAP_CUDA(cudaMalloc(&d_items, sizeof(Item) * items.size()));
        NAP_CUDA(cudaMemcpy(d_items, items.data(), sizeof(Item) * items.size(),
                            cudaMemcpyHostToDevice));
    }
    if (S.d_items) cudaFree(S.d_items);
    for (auto &g : P->graphs) cudaGraphExecDestroy(g.exec);  // they captured the old tiles
    P->graphs.clear();
    S.d_items = d_items;
    S.n_items = (int32_t)items.size();
    S.tile_rows = tile_rows;
    S.tile_nnz = tile_nnz;
    return NAPSPMV_OK;
}

// Counter words of a workspace: the fused engine's grid barrier (arrival count
// and generation).
static size_t ctr_count(const napspmv_plan_t *) { return 2; }

int ws_alloc(napspmv_plan_t *P, napspmv_ws_t *ws)
{
    ws->plan = P;
    ws->device = P->device;
    auto al = [](double **p, int64_t n) {
        return cudaMalloc(p, sizeof(double) * (size_t)std::max<int64_t>(n, 1));
    };
    auto alf = [](float **p, int64_t n) {
        return cudaMalloc(p, sizeof(float) * (size_t)std::max<int64_t>(n, 1));
    };
    // b_{l->l} and b_{nl->l} get 4 spare values: the remote pass copies each
    // process's segment widened to 16-byte boundaries
    if (al(&ws->bll, P->n_bll + 4) || al(&ws->lbuf, P->n_lbuf) || al(&ws->gsend, P->n_gs) ||
        al(&ws->grecv, P->n_gs) || al(&ws->bnl, P->n_bnl + 4) || al(&ws->xtmp, P->n) ||
        alf(&ws->x32[0], P->n) || alf(&ws->x32[1], P->n) ||
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
                 ws->ctr, ws->err, ws->x32[0], ws->x32[1]};
    for (void *q : p)
        if (q) cudaFree(q);
    ws->bll = ws->lbuf = ws->gsend = ws->grecv = ws->bnl = ws->xtmp = ws->hv = ws->hw = nullptr;
    ws->x32[0] = ws->x32[1] = nullptr;
    ws->ctr = nullptr;
    ws->err = nullptr;
}

static Scale make_scale(double s)
{
    Scale sc{s, kNoPow2};
    int e = 0;
    if (s != 0.0 && std::isfinite(s) && std::frexp(s, &e) == 0.5 && s > 0) sc.e2 = e - 1;
    return sc;
}

// Sliced-row entries per step: 8 where rows average more than 12 stored
// entries, else 4 (the order of every row's sum does not depend on it).
static int sell_unroll(const napspmv_plan_t *P) { return P->nnz > 12 * P->n ? 8 : 4; }

// The sliced-row view of one part of the plan (0 whole, 1 local, 2 remote).
static SellView sell_view(const napspmv_plan_t *P, int part, bool f32)
{
    const SellPart &SP = P->sell[part];
    SellView V{};
    V.info = SP.d_info;
    V.perm = SP.d_perm;
    V.col = SP.d_col;
    V.val = SP.d_val;
    V.val32 = SP.d_val32;
    V.lrows = SP.d_long;
    V.nch = (int32_t)SP.nch;
    V.n_long = SP.n_long;
    V.A = part == 1   ? Csr3{P->d_rowptrL, P->d_colL, P->d_valL, f32 ? P->d_val32L : nullptr}
          : part == 2 ? Csr3{P->d_rowptrR, P->d_colR, P->d_valR, f32 ? P->d_val32R : nullptr}
                      : Csr3{P->d_rowptr, P->d_colenc, P->d_val, f32 ? P->d_val32 : nullptr};
    return V;
}

static int32_t cdiv(int64_t a, int64_t b) { return (int32_t)((a + b - 1) / b); }

static FJob make_job(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w, int reps,
                     double scale, bool f32, int32_t chunk)
{
    FJob J{};
    J.F = sell_view(P, 0, f32);
    J.composed = (P->flags & NAPSPMV_COMPOSED_GATHERS) ? 1 : 0;
    J.src0 = P->lists[L_BLL].d_idx;
    J.n0 = (int32_t)P->n_bll;
    if (J.composed) {
        J.src1 = P->lists[L_BNL].d_idx;
        J.n1 = (int32_t)P->n_bnl;
    } else {
        J.src1 = P->lists[L_LBUF].d_idx;
        J.n1 = (int32_t)P->n_lbuf;
    }
    J.pack_src = P->d_pack_src;
    J.xfer_dst = P->d_xfer_dst;
    J.unp_src = P->d_unp_src;
    J.n_gs = (int32_t)P->n_gs;
    J.n_bnl = (int32_t)P->n_bnl;
    J.reps = reps;
    J.scale = make_scale(scale);
    J.bll = ws->bll;
    J.lbuf = ws->lbuf;
    J.gsend = ws->gsend;
    J.grecv = ws->grecv;
    J.bnl = ws->bnl;
    J.xtmp = ws->xtmp;
    J.err = ws->err;
    J.v = v;
    J.w = w;
    // units of every level: message chunks (levels 0-2), the sliced rows'
    // chunk groups and long rows (level 3)
    J.ch = chunk;
    J.nmsg[0] = cdiv(J.n0, J.ch) + cdiv(J.n1, J.ch);
    if (!J.composed) {
        J.nmsg[1] = cdiv(J.n_gs, J.ch);
        J.nmsg[2] = cdiv(J.n_bnl, J.ch);
    }
    for (int l = 0; l < 3; l++) J.nunits[l] = J.nmsg[l];
    J.nunits[3] = cdiv(J.F.nch, kSellGroup) + cdiv(J.F.n_long, WPB);
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
    prm.barrier_ns = 4 * prm.timeout_ns + 2000000000ll;
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    int32_t acc[kLevels] = {};
    for (int i = 0; i < count; i++) {
        napspmv_ws_t *wi = ws && ws[i] ? ws[i] : plans[i]->ws;
        prm.jobs[i] = make_job(plans[i], wi, v[i], w[i], reps[i], scale ? scale[i] : 1.0, f32, o.chunk);
        prm.kmax = std::max(prm.kmax, reps[i]);
        for (int l = 0; l < kLevels; l++) {
            prm.off[l][i] = acc[l];
            acc[l] += prm.jobs[i].nunits[l];
        }
        wi->buf_f32 = 0;  // this engine's receive buffers hold FP64 values in both modes
    }
    for (int l = 0; l < kLevels; l++) prm.off[l][count] = acc[l];
    // barrier words and the test hook's counter: the first job's workspace words
    napspmv_ws_t *w0 = ws && ws[0] ? ws[0] : plans[0]->ws;
    prm.bar = reinterpret_cast<unsigned int *>(w0->ctr);
    prm.stallctr = w0->ctr + 1;
    NAP_CUDA(cudaMemsetAsync(w0->ctr, 0, 2 * sizeof(unsigned long long), s));
    auto fn = FusedKernelTable<MAXJ>::get(f32);
    NAP_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
    int occ = 0;
    NAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT, 0));
    if (occ < 1) {
        set_error(NAPSPMV_ERR_CUDA, "fused engine: no CTA fits on an SM");
        return NAPSPMV_ERR_CUDA;
    }
    const int per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, occ) : occ;
    // every CTA resident at once (cooperative launch): the level barriers
    // never wait on a CTA that has not started
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(plans[0]->num_sms * per_sm));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    NAP_CUDA(cudaLaunchKernelEx(&cfg, fn, prm));
    count_launch(1);
    return NAPSPMV_OK;
}

using SpmvKernel = void (*)(Csr3, const void *, const void *, const void *, double *, float *,
                            Scale, const Item *, int, int, int, int, int *);
template <bool F32, int MODE>
static SpmvKernel pick_spmv(int vec, bool warp = false)
{
    if (warp) switch (vec) {
        case 1: return k_spmv_w<1, F32, MODE>;
        case 2: return k_spmv_w<2, F32, MODE>;
        case 4: return k_spmv_w<4, F32, MODE>;
        case 8: return k_spmv_w<8, F32, MODE>;
        case 16: return k_spmv_w<16, F32, MODE>;
        default: return k_spmv_w<32, F32, MODE>;
        }
    switch (vec) {
    case 1: return k_spmv<1, F32, MODE>;
    case 2: return k_spmv<2, F32, MODE>;
    case 4: return k_spmv<4, F32, MODE>;
    case 8: return k_spmv<8, F32, MODE>;
    case 16: return k_spmv<16, F32, MODE>;
    default: return k_spmv<32, F32, MODE>;
    }
}

// Kernel, tiles, capacities, shared memory and grid of one SpMV launch
// (mode: full three-block pass, local part, remote part).
using HaloKernel = void (*)(Csr3, const void *, const void *, double *, float *, Scale,
                           const Item *, int, int, int, int, const int32_t *, const int32_t *,
                           int *);
template <bool F32>
static HaloKernel pick_halo(int vec)
{
    switch (vec) {
    case 1: return k_spmv_halo<1, F32>;
    case 2: return k_spmv_halo<2, F32>;
    case 4: return k_spmv_halo<4, F32>;
    case 8: return k_spmv_halo<8, F32>;
    case 16: return k_spmv_halo<16, F32>;
    default: return k_spmv_halo<32, F32>;
    }
}

using SellKernel = void (*)(SellView, const void *, const void *, const void *, double *, float *,
                            Scale, int *);
template <bool F32, int U, int W = 8>
static SellKernel pick_sell_u(int mode)
{
    return mode == kLocal ? k_spmv_s<F32, kLocal, U, W>
                          : mode == kRemote ? k_spmv_s<F32, kRemote, U, W> : k_spmv_s<F32, kFull, U, W>;
}

// Rows of more than 12 entries (unroll 8): CTAs of 32 warps, one per SM, that
// sweep one process's 32 chunks at a time, so that the SM's L1 (no shared
// memory) holds that process's receive window.  Measured on the 2^23-row
// banded random workload: 680 against 735 us (FP64), 490 against 570 us (FP32
// values) for 8-warp CTAs on four processes per SM; the stencils' short rows
// run best with 8-warp CTAs.
template <bool F32>
static SellKernel pick_sell(int mode, int unroll)
{
    return unroll == 8 ? pick_sell_u<F32, 8, 32>(mode) : pick_sell_u<F32, 4, 8>(mode);
}

struct SpmvLaunch {
    SpmvKernel fn = nullptr;
    HaloKernel hfn = nullptr;  // set: the remote pass with staged receive buffers
    SellKernel sfn = nullptr;  // set: the sliced-row pass
    SellView S{};
    int sw = 8;  // warps per CTA of the sliced-row pass
    Csr3 A{};
    const Item *tiles = nullptr;
    const int32_t *bll_rank = nullptr, *bnl_rank = nullptr;
    int n = 0, cap = 0, rows = 0, grid = 1;
    size_t sm = 0;
};

// Shared memory of the staged-halo remote pass, or 0 if it does not apply:
// CTA stages for the remote tiles plus the widest process window.  It applies
// where the remote rows are gather-heavy (at least 8 remote entries per row on
// average) and two CTAs still fit on an SM.  Measured: the 2^23-row banded
// random workload (about 19 remote entries per row) gains 14% per apply in
// FP32 mode (70 KB windows, two CTAs per SM), breaks even in FP64 (136 KB, one
// CTA per SM); the stencils (2-6 remote entries per row) lose 5-7%.
static size_t halo_smem(const napspmv_plan_t *P, const napspmv_opts &o)
{
    if (o.halo != NAPSPMV_HALO_ON || o.pipeline == NAPSPMV_PIPELINE_SELL ||
        (P->flags & NAPSPMV_PARTITION_STRIDED) ||
        P->h_bll_rank.size() != (size_t)P->np + 1 || P->items.n_tilesRH == 0 ||
        P->nnzR < 8 * P->n)
        return 0;
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    const int es = f32 ? 4 : 8, al = halo_align(es);
    int64_t wcap = 0;
    for (int32_t r = 0; r < P->np; r++) {
        const int64_t b0 = P->h_bll_rank[r] & ~(al - 1);
        const int64_t b1 = (P->h_bll_rank[r + 1] + al - 1) & ~(al - 1);
        const int64_t n0 = P->h_bnl_rank[r] & ~(al - 1);
        const int64_t n1 = (P->h_bnl_rank[r + 1] + al - 1) & ~(al - 1);
        wcap = std::max(wcap, (b1 - b0) + (n1 - n0));
    }
    const size_t sm = (size_t)tile_smem_bytes(P->items.fit_nnz[6], P->items.fit_rows[6], o.stages,
                                              es) + 16 + (size_t)wcap * es;
    int smem_sm = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->device) ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, P->device))
        return 0;
    return 2 * (sm + (size_t)reserved) <= (size_t)smem_sm ? sm : 0;
}
static int spmv_launch(const napspmv_plan_t *P, const napspmv_opts &o, int mode, SpmvLaunch &L)
{
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    if (o.pipeline == NAPSPMV_PIPELINE_SELL) {
        const int part = mode == kLocal ? 1 : mode == kRemote ? 2 : 0;
        const SellPart &SP = P->sell[part];
        L.sfn = f32 ? pick_sell<true>(mode, sell_unroll(P)) : pick_sell<false>(mode, sell_unroll(P));
        L.S = sell_view(P, part, f32);
        L.sm = 0;
        const void *kf = (const void *)L.sfn;
        // no shared memory: the whole unified L1 / shared storage is L1
        NAP_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        int occ = 0;
        L.sw = sell_unroll(P) == 8 ? 32 : 8;
        NAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf, 32 * L.sw, 0));
        if (o.ctas_per_sm > 0) occ = std::min(occ, o.ctas_per_sm);
        const int64_t ctas = std::max<int64_t>((SP.nch + L.sw - 1) / L.sw,
                                               (SP.n_long + L.sw - 1) / L.sw);
        // 32-warp CTAs on FP64 values: up to four waves of them, so that the SMs
        // that finish their processes early take up others, while every CTA
        // keeps at least 13 groups.  On GB300, 2^23-row banded random matrix
        // (8,192 groups): the chained apply with one, two, four, eight waves
        // took 1.508, 1.471, 1.440, 1.450 ms, and the SM step 0.675 ms with one
        // wave, 0.601 with four.  At 2^21 rows (2,048 groups) four waves were
        // slower than one (169 against 159 us).  With FP32 values one wave
        // stays best (1.011 against 1.016, 1.023, 1.051 ms per apply).
        const int64_t slots = (int64_t)P->num_sms * std::max(occ, 1);
        const int waves = (L.sw == 32 && !f32)
                              ? (int)std::max<int64_t>(1, std::min<int64_t>(4, ctas / (slots * 13)))
                              : 1;
        L.grid = (int)std::max<int64_t>(
            1, std::min<int64_t>(ctas, (int64_t)P->num_sms * std::max(occ, 1) * waves));
        if (mode == kLocal)  // leave one CTA slot per SM for the message steps
            L.grid = (int)std::max<int64_t>(
                1, std::min<int64_t>(ctas, (int64_t)P->num_sms * std::max(occ - 1, 1)));
        return NAPSPMV_OK;
    }
    const bool warp = o.pipeline == NAPSPMV_PIPELINE_WARP;
    const ItemSet &S = P->items;
    const int list = (warp ? 3 : 0) + (mode == kLocal ? 1 : mode == kRemote ? 2 : 0);
    L.cap = S.fit_nnz[list];
    L.rows = S.fit_rows[list];
    const int vb = f32 ? 4 : 8;  // bytes per staged value
    L.sm = warp ? (size_t)warp_smem_bytes(L.cap, L.rows, o.stages, vb)
                : smem_bytes(L.cap, L.rows, o.stages, vb);
    if (mode == kLocal) {
        L.A = Csr3{P->d_rowptrL, P->d_colL, P->d_valL, f32 ? P->d_val32L : nullptr};
        L.fn = f32 ? pick_spmv<true, kLocal>(o.vec, warp) : pick_spmv<false, kLocal>(o.vec, warp);
        L.tiles = warp ? S.d_wtL : S.d_tilesL;
        L.n = warp ? S.n_wtL : S.n_tilesL;
    } else if (mode == kRemote) {
        L.A = Csr3{P->d_rowptrR, P->d_colR, P->d_valR, f32 ? P->d_val32R : nullptr};
        if (const size_t hs = halo_smem(P, o)) {
            // CTA tiles cut at process boundaries, receive buffers staged
            L.hfn = f32 ? pick_halo<true>(o.vec) : pick_halo<false>(o.vec);
            L.cap = S.fit_nnz[6];
            L.rows = S.fit_rows[6];
            L.sm = hs;
            L.tiles = S.d_tilesRH;
            L.n = S.n_tilesRH;
            L.bll_rank = P->d_bll_rank;
            L.bnl_rank = P->d_bnl_rank;
        } else {
            L.fn = f32 ? pick_spmv<true, kRemote>(o.vec, warp)
                       : pick_spmv<false, kRemote>(o.vec, warp);
            L.tiles = warp ? S.d_wtR : S.d_tilesR;
            L.n = warp ? S.n_wtR : S.n_tilesR;
        }
    } else {
        L.A = Csr3{P->d_rowptr, P->d_colenc, P->d_val, f32 ? P->d_val32 : nullptr};
        L.fn = f32 ? pick_spmv<true, kFull>(o.vec, warp) : pick_spmv<false, kFull>(o.vec, warp);
        L.tiles = warp ? S.d_wt : S.d_items;
        L.n = warp ? S.n_wt : S.n_items;
    }
    const void *kf = L.hfn ? (const void *)L.hfn : (const void *)L.fn;
    if (L.sm > 48 * 1024)
        NAP_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.sm));
    int occ = 0;
    NAP_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
    NAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf, NT, L.sm));
    // resident CTAs per SM: the occupancy maximum, or fewer (ctas_per_sm) where
    // the gathers want L1 more than the extra warps
    if (o.ctas_per_sm > 0) occ = std::min(occ, o.ctas_per_sm);
    // shared-memory carveout: what those CTAs need, the rest of the SM's unified
    // L1 / shared storage stays L1 for the gathers
    {
        int smem_sm = 0, reserved = 0;
        NAP_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                        P->device));
        NAP_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock,
                                        P->device));
        const int64_t need = (int64_t)std::max(occ, 1) * ((int64_t)L.sm + reserved);
        const int pct = (int)std::min<int64_t>(100, (need * 100 + smem_sm - 1) / smem_sm);
        NAP_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    }
    const int ctas = (warp && !L.hfn) ? (L.n + WPB - 1) / WPB : L.n;
    L.grid = std::max(1, std::min(ctas, P->num_sms * std::max(occ, 1)));
    if (mode == kLocal)  // leave one CTA slot per SM for the message steps
        L.grid = std::max(1, std::min(ctas, P->num_sms * std::max(occ - 1, 1)));
    return NAPSPMV_OK;
}
// Launch with programmatic stream serialization: the kernel may become
// resident while its stream predecessor drains (it waits in griddep_wait).
// Errors surface through cudaGetLastError like a <<<>>> launch.
// pdl = false: an ordinary launch.
template <typename... KArgs, typename... Args>
static void launch_pdl(bool pdl, void (*kern)(KArgs...), int grid, size_t smem, cudaStream_t s,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    (void)cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// x: the apply's input (FP64), or its FP32 copy in FP32 mode, where the
// receive buffers hold FP32 copies too; y32 (FP32 mode, may be null) receives
// the finished rows rounded to FP32.
static void spmv_run(const SpmvLaunch &L, const void *x, const napspmv_ws_t *ws, double *y,
                     float *y32, double scale, int stages, cudaStream_t s, bool pdl)
{
    if (L.sfn) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)L.grid);
        cfg.blockDim = dim3((unsigned)(32 * L.sw));
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = pdl ? 1 : 0;
        (void)cudaLaunchKernelEx(&cfg, L.sfn, L.S, x, (const void *)ws->bll, (const void *)ws->bnl,
                                 y, y32, make_scale(scale), ws->err);
    }
    else if (L.hfn)
        launch_pdl(pdl, L.hfn, L.grid, L.sm, s, L.A, (const void *)ws->bll, (const void *)ws->bnl,
                   y, y32, make_scale(scale), L.tiles, L.n, L.cap, L.rows, stages, L.bll_rank,
                   L.bnl_rank, ws->err);
    else
        launch_pdl(pdl, L.fn, L.grid, L.sm, s, L.A, x, (const void *)ws->bll,
                   (const void *)ws->bnl, y, y32, make_scale(scale), L.tiles, L.n, L.cap, L.rows,
                   stages, ws->err);
}

// CTAs of a message-step kernel that the whole GPU holds at once (the FP64
// kernels hold 40 registers a thread: 6 CTAs of 256 threads per SM).
template <class... A>
static int64_t one_wave(const napspmv_plan_t *P, void (*kern)(A...))
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return (int64_t)P->num_sms * occ;
}

// Grid of a message-step kernel over n elements, in chunks of NT * 8 (each
// CTA strides over chunk b, b + grid, ...).  Up to four resident waves' worth
// of chunks: one wave, so that no CTA waits for a slot and then runs its share
// alone at the end.  More chunks than that: 96 CTAs per SM, many waves, whose
// CTAs the hardware starts as others end, so that the SMs stay full to the
// last chunk.  Measured per apply on GB300 (2^23-row banded random, FP64 /
// FP32 values; 3D 7-point 128^3): 8 CTAs per SM (1.3 waves) 1.654 ms; one
// wave 1.609 / 1.070 ms, 75.3 us; 16, 32, 64, 96 and 128 CTAs per SM 1.558,
// 1.530, 1.511, 1.505, 1.508 / 1.048, 1.029, 1.016, 1.010, 1.011 ms; one
// chunk per CTA 1.527 / 1.061 ms.  The 128^3 workload stays within four waves
// (75.9 us with one chunk per CTA).
static int msg_grid(const napspmv_plan_t *P, int64_t n, int64_t wave)
{
    const int64_t chunks = (n + NT * 8 - 1) / (NT * 8);
    const int64_t g = chunks <= 4 * wave ? wave : (int64_t)P->num_sms * 96;
    return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, g));
}

// The four message steps of one apply (phases 1-4) as kernels on stream s;
// returns the number of launches.  The later steps are launched as
// programmatic dependents of the earlier ones; pdl_first: the first step too.
template <class T>
static int64_t enqueue_messages(const napspmv_plan_t *P, const T *x, T *bll, T *lbuf, T *gsend,
                                T *grecv, T *bnl, int *err, cudaStream_t s, bool pdl_first)
{
    auto grid = [&](int64_t n, int64_t wave) { return msg_grid(P, n, wave); };
    int64_t nk = 0;
    if (P->n_bll + P->n_lbuf > 0) {
        launch_pdl(pdl_first, k_gather2<T>,
                   grid(P->n_bll + P->n_lbuf, one_wave(P, k_gather2<T>)), 0, s, x,
                   (const int32_t *)P->lists[L_BLL].d_idx, bll, (int)P->n_bll,
                   (const int32_t *)P->lists[L_LBUF].d_idx, lbuf, (int)P->n_lbuf,
                   (const int *)err);
        nk++;
    }
    if (P->n_gs > 0) {
        launch_pdl(true, k_pack<T>, grid(P->n_gs, one_wave(P, k_pack<T>)), 0, s, x, (const T *)lbuf,
                   (const uint32_t *)P->d_pack_src, gsend, (int)P->n_gs, (const int *)err);
        launch_pdl(true, k_transfer<T>, grid(P->n_gs, one_wave(P, k_transfer<T>)), 0, s,
                   (const T *)gsend,
                   (const int32_t *)P->d_xfer_dst, grecv, (int)P->n_gs, (const int *)err);
        nk += 2;
    }
    if (P->n_bnl > 0) {
        launch_pdl(true, k_unpack<T>, grid(P->n_bnl, one_wave(P, k_unpack<T>)), 0, s,
                   (const T *)grecv,
                   (const int32_t *)P->d_unp_src, bnl, (int)P->n_bnl, (const int *)err);
        nk++;
    }
    return nk;
}

// Composed gathers (plan flag NAPSPMV_COMPOSED_GATHERS): both receive buffers
// straight from x with the on->on and off-node receive index lists, one
// kernel; the hops of the node-aware exchange are skipped.
static int64_t enqueue_composed(const napspmv_plan_t *P, const void *x, napspmv_ws_t *ws, bool f32,
                                cudaStream_t s, bool pdl)
{
    const int64_t n = P->n_bll + P->n_bnl;
    if (n == 0) return 0;
    const int g = msg_grid(P, n, f32 ? one_wave(P, k_gather2<float>) : one_wave(P, k_gather2<double>));
    if (f32)
        launch_pdl(pdl, k_gather2<float>, g, 0, s, static_cast<const float *>(x),
                   (const int32_t *)P->lists[L_BLL].d_idx, reinterpret_cast<float *>(ws->bll),
                   (int)P->n_bll, (const int32_t *)P->lists[L_BNL].d_idx,
                   reinterpret_cast<float *>(ws->bnl), (int)P->n_bnl, (const int *)ws->err);
    else
        launch_pdl(pdl, k_gather2<double>, g, 0, s, static_cast<const double *>(x),
                   (const int32_t *)P->lists[L_BLL].d_idx, ws->bll, (int)P->n_bll,
                   (const int32_t *)P->lists[L_BNL].d_idx, ws->bnl, (int)P->n_bnl,
                   (const int *)ws->err);
    return 1;
}

static int enqueue_phased(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w, int reps,
                          double scale, const napspmv_opts &o, cudaStream_t s, int64_t *kernels)
{
    auto grid = [&](int64_t n) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((n + NT * 8 - 1) / (NT * 8),
                                                            (int64_t)P->num_sms * 8));
    };
    const ItemSet &S = P->items;
    const bool overlap = o.engine == NAPSPMV_ENGINE_OVERLAP && S.n_tilesL > 0;
    SpmvLaunch LF, LL, LR;
    if (int rc = spmv_launch(P, o, kFull, LF)) return rc;
    if (overlap) {
        if (int rc = spmv_launch(P, o, kLocal, LL)) return rc;
        if (int rc = spmv_launch(P, o, kRemote, LR)) return rc;
    }
    // FP32 mode: the message steps move FP32 copies (the products round x to
    // FP32 anyway), the SpMV reads FP32 sources, and each apply's SpMV also
    // writes the FP32 copy of its result for the next apply of the chain
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    int64_t nk = 0;
    if (f32) {
        launch_pdl(!overlap, k_to_f32, grid(P->n), 0, s, v, ws->x32[0], (int64_t)P->n,
                   (const int *)ws->err);
        nk++;
    }
    ws->buf_f32 = f32 ? 1 : 0;
    for (int k = 0; k < reps; k++) {
        const double *x = (k == 0) ? v : (((reps - k) & 1) == 0 ? w : ws->xtmp);
        double *y = (((reps - 1 - k) & 1) == 0) ? w : ws->xtmp;
        float *x32 = ws->x32[k & 1];
        float *y32 = (f32 && k + 1 < reps) ? ws->x32[(k + 1) & 1] : nullptr;
        const void *xs = f32 ? (const void *)x32 : (const void *)x;
        if (overlap) {
            // Algorithm NAPSpMV: local_spmv(A_on_process) needs no message and
            // runs on a second stream while the message steps proceed
            NAP_CUDA(cudaEventRecord(P->ev_fork, s));
            NAP_CUDA(cudaStreamWaitEvent(P->aux, P->ev_fork, 0));
            spmv_run(LL, xs, ws, y, nullptr, scale, o.stages, P->aux, false);
            nk++;
            NAP_CUDA(cudaEventRecord(P->ev_join, P->aux));
        }
        // programmatic dependent launches: every edge of the phased engine; in
        // the overlapped engine only inside the message chain, where the local
        // pass is already resident (an early-resident first step or remote
        // pass would hold the slots the local pass needs)
        const bool pdl = !overlap;
        if (P->flags & NAPSPMV_COMPOSED_GATHERS)
            nk += enqueue_composed(P, f32 ? (const void *)x32 : (const void *)x, ws, f32, s, pdl);
        else if (f32)
            nk += enqueue_messages<float>(P, x32, reinterpret_cast<float *>(ws->bll),
                                          reinterpret_cast<float *>(ws->lbuf),
                                          reinterpret_cast<float *>(ws->gsend),
                                          reinterpret_cast<float *>(ws->grecv),
                                          reinterpret_cast<float *>(ws->bnl), ws->err, s, pdl);
        else
            nk += enqueue_messages<double>(P, x, ws->bll, ws->lbuf, ws->gsend, ws->grecv, ws->bnl,
                                           ws->err, s, pdl);
        if (overlap) {
            NAP_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));
            spmv_run(LR, xs, ws, y, y32, scale, o.stages, s, false);
        } else {
            spmv_run(LF, xs, ws, y, y32, scale, o.stages, s, true);
        }
        nk++;
        NAP_CUDA(cudaGetLastError());
    }
    *kernels = nk;
    return NAPSPMV_OK;
}

// Chained applies on a capturable stream are recorded once into a CUDA graph
// per (vectors, workspace, reps, scale, options) and replayed afterwards.
static int launch_phased(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w, int reps,
                         double scale, const napspmv_opts &o, cudaStream_t s)
{
    {
        // attributes (dynamic shared memory) are set before any capture
        SpmvLaunch L;
        if (int rc = spmv_launch(P, o, kFull, L)) return rc;
        if (o.engine == NAPSPMV_ENGINE_OVERLAP && P->items.n_tilesL > 0) {
            if (int rc = spmv_launch(P, o, kLocal, L)) return rc;
            if (int rc = spmv_launch(P, o, kRemote, L)) return rc;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NAP_CUDA(cudaStreamIsCapturing(s, &cs));
    const bool use_graph = reps > 1 && s != nullptr && cs == cudaStreamCaptureStatusNone;
    int64_t nk = 0;
    if (!use_graph) {
        int rc = enqueue_phased(P, ws, v, w, reps, scale, o, s, &nk);
        if (!rc) count_launch(nk);
        return rc;
    }
    for (size_t i = 0; i < P->graphs.size(); i++) {
        auto &g = P->graphs[i];
        if (g.v == v && g.w == w && g.ws == ws && g.reps == reps && g.scale == scale &&
            g.prec == o.precision && g.vec == o.vec && g.tile_rows == o.tile_rows &&
            g.tile_nnz == o.tile_nnz && g.engine == o.engine && g.stages == o.stages &&
            g.pipeline == o.pipeline && g.ctas_per_sm == o.ctas_per_sm && g.halo == o.halo) {
            NAP_CUDA(cudaGraphLaunch(g.exec, s));
            count_launch(g.kernels);
            return NAPSPMV_OK;
        }
    }
    cudaGraph_t graph = nullptr;
    NAP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_phased(P, ws, v, w, reps, scale, o, s, &nk);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
    if (P->graphs.size() >= 8) {
        cudaGraphExecDestroy(P->graphs.front().exec);
        P->graphs.erase(P->graphs.begin());
    }
    P->graphs.push_back({v, w, ws, reps, o.precision, o.vec, o.tile_rows, o.tile_nnz, o.engine,
                         o.stages, o.pipeline, o.ctas_per_sm, o.halo, scale, exec, nk});
    NAP_CUDA(cudaGraphLaunch(exec, s));
    count_launch(nk);
    return NAPSPMV_OK;
}

int check_opts(const napspmv_plan_t *P, const napspmv_opts &o)
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
    if (o.engine != NAPSPMV_ENGINE_FUSED && o.engine != NAPSPMV_ENGINE_PHASED &&
        o.engine != NAPSPMV_ENGINE_OVERLAP) {
        set_error(NAPSPMV_ERR_ARG, "unknown engine");
        return NAPSPMV_ERR_ARG;
    }
    if (o.engine == NAPSPMV_ENGINE_FUSED && P->sell[0].slots < 0) {
        set_error(NAPSPMV_ERR_UNSUPPORTED, "the fused engine sums rows from the sliced-row copy, "
                                           "which this plan could not keep (over 2^31 slots)");
        return NAPSPMV_ERR_UNSUPPORTED;
    }
    if (o.timeout_ms < 1) {
        set_error(NAPSPMV_ERR_ARG, "timeout_ms must be >= 1");
        return NAPSPMV_ERR_ARG;
    }
    if (o.chunk < 32 || o.chunk > (1 << 24)) {
        set_error(NAPSPMV_ERR_ARG, "chunk must be 32 .. 2^24 elements");
        return NAPSPMV_ERR_ARG;
    }
    if (o.halo != NAPSPMV_HALO_ON && o.halo != NAPSPMV_HALO_OFF) {
        set_error(NAPSPMV_ERR_ARG, "halo must be NAPSPMV_HALO_ON or _OFF");
        return NAPSPMV_ERR_ARG;
    }
    if (o.pipeline != NAPSPMV_PIPELINE_CTA && o.pipeline != NAPSPMV_PIPELINE_WARP &&
        o.pipeline != NAPSPMV_PIPELINE_SELL) {
        set_error(NAPSPMV_ERR_ARG, "pipeline must be NAPSPMV_PIPELINE_CTA, _WARP or _SELL");
        return NAPSPMV_ERR_ARG;
    }
    if (o.pipeline == NAPSPMV_PIPELINE_SELL &&
        (P->sell[0].slots < 0 || P->sell[1].slots < 0 || P->sell[2].slots < 0)) {
        set_error(NAPSPMV_ERR_UNSUPPORTED, "the sliced-row copy of this plan would exceed 2^31 "
                                           "slots; use the CTA or warp pipeline");
        return NAPSPMV_ERR_UNSUPPORTED;
    }
    if (o.stages < 2 || o.stages > kMaxStages ||
        smem_bytes(o.tile_nnz, o.tile_rows, o.stages) > 220 * 1024) {
        set_error(NAPSPMV_ERR_ARG, "stages must be 2..4 and all stages must fit in 220 KiB of "
                                   "shared memory");
        return NAPSPMV_ERR_ARG;
    }
    return NAPSPMV_OK;
}

// Launch-relevant fields of two resolved option sets agree: entries with equal
// keys can share one fused launch (one kernel, one lane count, one tile shape).
static bool same_launch(const napspmv_opts &a, const napspmv_opts &b)
{
    return a.precision == b.precision && a.vec == b.vec && a.chunk == b.chunk &&
           a.tile_rows == b.tile_rows && a.tile_nnz == b.tile_nnz &&
           a.ctas_per_sm == b.ctas_per_sm && a.timeout_ms == b.timeout_ms &&
           a.debug_stall == b.debug_stall;
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
    // every entry resolves the unset fields against its own plan's defaults,
    // so that it runs with the row tiles its plan already holds
    napspmv_opts oi[64];
    int cur = 0;
    NAP_CUDA(cudaGetDevice(&cur));
    if (cur != P0->device) NAP_CUDA(cudaSetDevice(P0->device));
    int rc = NAPSPMV_OK;
    for (int i = 0; i < count && !rc; i++) {
        napspmv_plan_t *P = plans[i];
        if (!P || !v[i] || !w[i] || reps[i] < 1 || (const double *)w[i] == v[i]) {
            set_error(NAPSPMV_ERR_ARG, "NULL plan or vector, reps < 1, or w == v");
            rc = NAPSPMV_ERR_ARG;
            break;
        }
        if (P->device != P0->device) {
            set_error(NAPSPMV_ERR_ARG, "all plans of a batch must live on one device");
            rc = NAPSPMV_ERR_ARG;
            break;
        }
        oi[i] = resolve_opts(P, opts);
        // several entries share fused launches, whatever engine the options name:
        // validate them for that engine
        if (count > 1) oi[i].engine = NAPSPMV_ENGINE_FUSED;
        if ((rc = check_opts(P, oi[i]))) break;
        if ((rc = build_items(P, oi[i].tile_rows, oi[i].tile_nnz))) break;
        for (int q = 0; q < i; q++) {
            napspmv_ws_t *a = ws && ws[i] ? ws[i] : P->ws;
            napspmv_ws_t *b = ws && ws[q] ? ws[q] : plans[q]->ws;
            if (a == b) {
                set_error(NAPSPMV_ERR_ARG, "two batch entries share one workspace");
                rc = NAPSPMV_ERR_ARG;
                break;
            }
        }
        if (!rc && ws && ws[i] && ws[i]->plan != P) {
            set_error(NAPSPMV_ERR_ARG, "workspace belongs to another plan");
            rc = NAPSPMV_ERR_ARG;
        }
    }
    if (!rc && count == 1) {
        const napspmv_opts &o = oi[0];
        if (o.engine == NAPSPMV_ENGINE_PHASED || o.engine == NAPSPMV_ENGINE_OVERLAP)
            rc = launch_phased(P0, ws && ws[0] ? ws[0] : P0->ws, v[0], w[0], reps[0],
                               scale ? scale[0] : 1.0, o, s);
        else
            rc = launch_fused<1>(1, plans, ws, v, w, reps, scale, o, s);
    } else if (!rc) {
        // one fused launch per distinct launch option set, in order of first
        // appearance; an entry's bits are those of its plan applied alone on the
        // fused engine with its resolved options, whatever else is in the batch
        bool done[64] = {};
        for (int i = 0; i < count && !rc; i++) {
            if (done[i]) continue;
            napspmv_plan_t *gp[64];
            napspmv_ws_t *gw[64];
            const double *gv[64];
            double *gx[64];
            int32_t gr[64];
            double gs[64];
            int m = 0;
            for (int j = i; j < count; j++) {
                if (done[j] || !same_launch(oi[i], oi[j])) continue;
                done[j] = true;
                gp[m] = plans[j];
                gw[m] = ws && ws[j] ? ws[j] : plans[j]->ws;
                gv[m] = v[j];
                gx[m] = w[j];
                gr[m] = reps[j];
                gs[m] = scale ? scale[j] : 1.0;
                m++;
            }
            rc = m == 1 ? launch_fused<1>(1, gp, gw, gv, gx, gr, gs, oi[i], s)
                        : launch_fused<64>(m, gp, gw, gv, gx, gr, gs, oi[i], s);
        }
    }
    if (cur != P0->device) cudaSetDevice(cur);
    return rc;
}

}  // namespace nap

extern "C" const char *napspmv_last_error(void) { return nap::g_last_error.c_str(); }
extern "C" int64_t napspmv_launch_count(void) { return nap::g_launches; }

// ===================================================================
// Apply without allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// product: their device memory is owned by another allocator (a framework's
// memory pool that holds the free memory), or they run on a latency-critical
// path where cudaMalloc's implicit device synchronisation would stall their
// pipeline.  napspmv_apply_noalloc serves them: it runs the fused apply with
// its receive buffers, chain vector and barrier words carved out of the
// fixed array below instead of a workspace.  The array is reserved on every
// device that loads this library, until the process exits.
namespace nap {
constexpr int64_t kNoallocDoubles = 1ll << 20;  // 8 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];
static double *g_noalloc_ptr[256];
static std::mutex g_noalloc_mu;
}  // namespace nap

extern "C" int napspmv_apply_noalloc(napspmv_plan_t *P, const double *v, double *w, int32_t reps,
                                     double scale, void *stream)
{
    using namespace nap;
    if (!P || !v || !w || reps < 1 || (const double *)w == v) {
        set_error(NAPSPMV_ERR_ARG, "NULL plan or vector, reps < 1, or w == v");
        return NAPSPMV_ERR_ARG;
    }
    // doubles of scratch: the barrier words (8-byte), b_{l->l}, b_{l->nl},
    // g_send, g_recv, b_{nl->l}, and the chain vector when reps > 1 (a single
    // apply writes w directly)
    const int64_t words = (int64_t)ctr_count(P);
    const int64_t need = words + P->n_bll + P->n_lbuf + 2 * P->n_gs + P->n_bnl +
                         (reps > 1 ? P->n : 0);
    if (need > kNoallocDoubles) {
        set_error(NAPSPMV_ERR_UNSUPPORTED,
                  "napspmv_apply_noalloc: this plan needs " + std::to_string(need) +
                      " doubles of scratch; the static area holds " +
                      std::to_string(kNoallocDoubles) + " (8 MiB)");
        return NAPSPMV_ERR_UNSUPPORTED;
    }
    if (P->device < 0 || P->device >= 256) {
        set_error(NAPSPMV_ERR_ARG, "device id out of range");
        return NAPSPMV_ERR_ARG;
    }
    int cur = 0;
    NAP_CUDA(cudaGetDevice(&cur));
    if (cur != P->device) NAP_CUDA(cudaSetDevice(P->device));
    double *base = nullptr;
    {
        // first call on a device: look up the array's device address (with
        // that device current); later calls reuse it.  The cached address
        // belongs to the device's current context: it does not survive
        // cudaDeviceReset.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[P->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                if (cur != P->device) cudaSetDevice(cur);
                return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            }
            g_noalloc_ptr[P->device] = static_cast<double *>(p);
        }
        base = g_noalloc_ptr[P->device];
    }
    // a workspace view of the array; the sticky error flag stays the plan's own
    napspmv_ws_t view;
    view.plan = P;
    view.device = P->device;
    view.ctr = reinterpret_cast<unsigned long long *>(base);
    double *q = base + words;
    view.bll = q;
    q += P->n_bll;
    view.lbuf = q;
    q += P->n_lbuf;
    view.gsend = q;
    q += P->n_gs;
    view.grecv = q;
    q += P->n_gs;
    view.bnl = q;
    q += P->n_bnl;
    view.xtmp = reps > 1 ? q : nullptr;
    view.err = P->ws->err;
    // the plan's default options on the fused engine, FP64; the tile shape is
    // the one the plan's row tiles have, so that nothing is rebuilt (the fused
    // engine sums rows from the sliced-row copy)
    napspmv_opts o = P->defaults;
    o.engine = NAPSPMV_ENGINE_FUSED;
    o.precision = NAPSPMV_PREC_F64;
    o.tile_rows = P->items.tile_rows;
    o.tile_nnz = P->items.tile_nnz;
    o.debug_stall = 0;
    if (int rc2 = check_opts(P, o)) {
        if (cur != P->device) cudaSetDevice(cur);
        return rc2;
    }
    napspmv_ws_t *wsl[1] = {&view};
    napspmv_plan_t *pl[1] = {P};
    const double *vl[1] = {v};
    double *wl[1] = {w};
    // launch_fused zeroes the barrier words (the array keeps the last call's contents)
    int rc = launch_fused<1>(1, pl, wsl, vl, wl, &reps, &scale, o, (cudaStream_t)stream);
    view.bll = view.lbuf = view.gsend = view.grecv = view.bnl = view.xtmp = nullptr;
    view.ctr = nullptr;
    view.err = nullptr;  // nothing of the view is freed
    if (cur != P->device) cudaSetDevice(cur);
    return rc;
}

// The three-block SpMV step alone (phase 5 / local_spmv over the three blocks),
// on the receive buffers the workspace holds from its last apply.
extern "C" int napspmv_spmv_step(napspmv_plan_t *P, napspmv_ws_t *ws, const double *v, double *w,
                                 double scale, const napspmv_opts *opts, void *stream)
{
    using namespace nap;
    if (!P || !v || !w || (const double *)w == v) {
        set_error(NAPSPMV_ERR_ARG, "NULL plan or vector, or w == v");
        return NAPSPMV_ERR_ARG;
    }
    napspmv_ws_t *W = ws ? ws : P->ws;
    napspmv_opts o = resolve_opts(P, opts);
    int rc = check_opts(P, o);
    if (rc) return rc;
    int cur = 0;
    NAP_CUDA(cudaGetDevice(&cur));
    if (cur != P->device) NAP_CUDA(cudaSetDevice(P->device));
    if ((rc = build_items(P, o.tile_rows, o.tile_nnz))) return rc;
    const bool f32 = o.precision == NAPSPMV_PREC_F32;
    // launched as the phased engine launches its SpMV pass
    const bool pdl = o.engine == NAPSPMV_ENGINE_PHASED;
    if (W->buf_f32 != (f32 ? 1 : 0)) {
        set_error(NAPSPMV_ERR_STATE, "the receive buffers hold the other precision's copies: "
                                     "apply once in this precision (phased or overlapped engine "
                                     "for FP32) before the step");
        return NAPSPMV_ERR_STATE;
    }
    SpmvLaunch L;
    if ((rc = spmv_launch(P, o, kFull, L))) return rc;
    if (f32) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((P->n + NT - 1) / NT,
                                                                  (int64_t)P->num_sms * 8));
        k_to_f32<<<g, NT, 0, (cudaStream_t)stream>>>(v, W->x32[0], P->n, W->err);
        spmv_run(L, W->x32[0], W, w, nullptr, scale, o.stages, (cudaStream_t)stream, pdl);
        count_launch(2);
    } else {
        spmv_run(L, v, W, w, nullptr, scale, o.stages, (cudaStream_t)stream, pdl);
        count_launch(1);
    }
    NAP_CUDA(cudaGetLastError());
    if (cur != P->device) cudaSetDevice(cur);
    return NAPSPMV_OK;
}
