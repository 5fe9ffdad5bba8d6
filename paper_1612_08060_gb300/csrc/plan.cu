// plan.cu -- GPU construction of the standard and node-aware communication
// plans and of the three-block CSR.
//
// Every set of the paper is obtained on the device as a sorted, de-duplicated
// array of packed 64-bit keys:
//   (r, t, j)  r = owner(j) sends column j to the row owner t   Eqs. P, D
//   (n, m, j)  node n sends column j to node m                  Eqs. N, E
//   (t, j)     receive layouts of rank t                        (b_{l->l}, b_{nl->l})
//   (p, s, j)  on_node -> off_node                              Eqs. L0, IL0
//   (q, s, j)  off_node -> on_node                              Eqs. L1, IL1
// built with CUB radix sort / select / run-length encode (library primitives
// for plan time only; the apply path is hand-written).  The per-node-pair
// process assignment T/U (Eqs. T, U and the mapping rule after them, the
// text's variant, or the majority mapping whose per-pair counts are taken on
// the device) is O(node pairs) and runs on the host.  The owner of a row or
// column follows the plan's partition: contiguous blocks (Eq. R) or strided
// (row i on process i mod n_p).  The plan also keeps the matrix split into its
// on_process and remote parts for the overlapped engine.
#include <cub/cub.cuh>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace nap {
namespace {

struct NapError {
    int code;
    std::string msg;
};

inline void ck(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw NapError{e == cudaErrorMemoryAllocation ? NAPSPMV_ERR_OOM : NAPSPMV_ERR_CUDA,
                       std::string(what) + ": " + cudaGetErrorString(e)};
    }
}
#define CK(x) ck((x), #x)

template <class T>
struct dvec {
    T *p = nullptr;
    int64_t n = 0;
    dvec() = default;
    explicit dvec(int64_t count) { alloc(count); }
    void alloc(int64_t count)
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = count;
        if (count > 0) CK(cudaMalloc(&p, sizeof(T) * (size_t)count));
    }
    ~dvec()
    {
        if (p) cudaFree(p);
    }
    T *release()
    {
        T *q = p;
        p = nullptr;
        return q;
    }
    dvec(const dvec &) = delete;
    dvec &operator=(const dvec &) = delete;
};

template <class T>
T *upload(const std::vector<T> &h)
{
    T *d = nullptr;
    size_t bytes = sizeof(T) * std::max<size_t>(h.size(), 1);
    CK(cudaMalloc(&d, bytes));
    if (!h.empty()) CK(cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return d;
}

constexpr uint64_t SENT = ~0ull;

inline int bits_for(int64_t maxval)  // bits to hold 0..maxval
{
    int b = 1;
    while (b < 63 && (int64_t(1) << b) <= maxval) b++;
    return b;
}

// Row partition: contiguous blocks of Eq. R (first N mod n_p ranks one row
// longer), or strided (row i on rank i mod n_p, Sec. 5).
struct Part {
    int64_t q, rem, big, np;
    bool strided;
    __host__ __device__ int64_t owner(int64_t j) const
    {
        if (strided) return j % np;
        return j < big ? j / (q + 1) : rem + (j - big) / q;
    }
    // first row of rank r (contiguous blocks only)
    __host__ __device__ int64_t start(int64_t r) const { return r * q + (r < rem ? r : rem); }
};

inline int blocks_for(int64_t n, int t = 256)
{
    int64_t b = (n + t - 1) / t;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

// ----------------------------------------------------------------- kernels

__global__ void k_check_rowptr(const int64_t *rp, int64_t n, int64_t nnz, int *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (rp[i + 1] < rp[i]) atomicOr(bad, 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(bad, 1);
}

__global__ void k_row_of(const int64_t *rp, int64_t n, const int32_t *col, int32_t *row_of,
                         int *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            row_of[k] = (int32_t)i;
            int32_t c = col[k];
            if (c < 0 || c >= n) atomicOr(bad, 2);
        }
    }
}

__global__ void k_pair_keys(const int32_t *row_of, const int32_t *col, int64_t nnz, int jb,
                            uint64_t *keys)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        keys[k] = ((uint64_t)row_of[k] << jb) | (uint32_t)col[k];
}

__global__ void k_adjacent_equal(const uint64_t *keys, int64_t n, int *bad)
{
    for (int64_t k = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        if (keys[k] == keys[k - 1]) atomicOr(bad, 4);
}

// Block of every stored entry (Eqs. on_proc, on_node, off_node) and the
// (r, t, j) key of every off-process entry.
__global__ void k_classify(const int32_t *row_of, const int32_t *col, int64_t nnz, Part part,
                           int32_t ppn, int rb, int jb, uint8_t *tag, uint64_t *key,
                           unsigned long long *blk_count)
{
    unsigned long long c[3] = {0, 0, 0};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = row_of[k], j = col[k];
        int64_t t = part.owner(i), r = part.owner(j);
        uint8_t b = (r == t) ? 0 : ((r / ppn == t / ppn) ? 1 : 2);
        tag[k] = b;
        c[b]++;
        key[k] = b ? (((uint64_t)r << (rb + jb)) | ((uint64_t)t << jb) | (uint64_t)j) : SENT;
    }
    for (int q = 0; q < 3; q++) {
        unsigned long long s = c[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(&blk_count[q], s);
    }
}

__global__ void k_shift(const uint64_t *in, int64_t n, int sh, uint64_t *out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = in[k] >> sh;
}

__global__ void k_low(const uint64_t *in, int64_t n, uint64_t mask, int32_t *out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (int32_t)(in[k] & mask);
}

// (r, t, j) -> (t, j)
__global__ void k_rekey_tj(const uint64_t *in, int64_t n, int rb, int jb, uint64_t *out)
{
    uint64_t rmask = (1ull << rb) - 1, jmask = (1ull << jb) - 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t t = (in[k] >> jb) & rmask;
        out[k] = (t << jb) | (in[k] & jmask);
    }
}

// (r, t, j) -> (node r, node t, j)
__global__ void k_rekey_node(const uint64_t *in, int64_t n, int rb, int jb, int nb, int32_t ppn,
                             uint64_t *out)
{
    uint64_t rmask = (1ull << rb) - 1, jmask = (1ull << jb) - 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = in[k] >> (rb + jb), t = (in[k] >> jb) & rmask;
        out[k] = ((r / ppn) << (nb + jb)) | ((t / ppn) << jb) | (in[k] & jmask);
    }
}

struct NotSent {
    __host__ __device__ bool operator()(uint64_t k) const { return k != SENT; }
};
struct SameNode {
    int rb, jb, ppn;
    bool want;
    __host__ __device__ bool operator()(uint64_t k) const
    {
        uint64_t r = k >> (rb + jb), t = (k >> jb) & ((1ull << rb) - 1);
        return ((r / ppn) == (t / ppn)) == want;
    }
};

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Content of g_send (INTER messages in (src, dst) order), its transfer
// destinations in g_recv, the message of every element and the J0 keys.
__global__ void k_fill_gsend(int64_t n_gs, const int64_t *gs_off, int64_t n_msg,
                             const int32_t *msg_pair, const int32_t *msg_src,
                             const int64_t *msg_gr, const int64_t *msg_lo,
                             const int32_t *node_ptr, const int32_t *node_idx, Part part, int rb,
                             int jb, int32_t *gs_j, int32_t *xfer_dst, int32_t *msg_of,
                             uint64_t *j0key)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_gs;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n_msg - 1;  // last message with gs_off <= e
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (gs_off[mid] <= e)
                lo = mid;
            else
                hi = mid - 1;
        }
        int32_t k = msg_pair[lo];
        int64_t off = e - gs_off[lo];
        int32_t j = node_idx[node_ptr[k] + msg_lo[lo] + off];
        gs_j[e] = j;
        xfer_dst[e] = (int32_t)(msg_gr[lo] + off);
        msg_of[e] = (int32_t)lo;
        int64_t s = msg_src[lo], p = part.owner(j);
        j0key[e] = (p != s) ? (((uint64_t)p << (rb + jb)) | ((uint64_t)s << jb) | (uint64_t)j)
                            : SENT;
    }
}

__global__ void k_pack_src(int64_t n_gs, const int32_t *gs_j, const int32_t *msg_of,
                           const int32_t *msg_src, const int32_t *lbuf_ptr, const int32_t *lbuf_j,
                           Part part, uint32_t *pack_src, int *bad)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_gs;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t j = gs_j[e], s = msg_src[msg_of[e]];
        if (part.owner(j) == s) {
            pack_src[e] = (uint32_t)j;
        } else {
            int64_t b = lbuf_ptr[s], len = lbuf_ptr[s + 1] - b;
            int64_t pos = lower_bound_i32(lbuf_j + b, len, j);
            if (pos >= len || lbuf_j[b + pos] != j) atomicOr(bad, 8);
            pack_src[e] = kFromLbuf | (uint32_t)(b + pos);
        }
    }
}

// Off-node receive entries (t, j): the receiving process q of j's node pair,
// the J1 key (q, t, j) when q != t, and the g_recv position to unpack from.
__global__ void k_unpack_src(int64_t n_bnl, const uint64_t *bnl_keys, int jb, Part part,
                             int32_t ppn, int nb, int64_t n_pairs, const uint64_t *pair_key,
                             const int64_t *pair_piece, const int64_t *piece_lo,
                             const int32_t *piece_dst, const int64_t *piece_gr,
                             const int32_t *node_ptr, const int32_t *node_idx, int rb,
                             uint64_t *j1key, int32_t *unp_src, int *bad)
{
    uint64_t jmask = (1ull << jb) - 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_bnl;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t t = bnl_keys[e] >> jb;
        int32_t j = (int32_t)(bnl_keys[e] & jmask);
        uint64_t nj = part.owner(j) / ppn, m = t / ppn;
        uint64_t pk = (nj << nb) | m;
        int64_t lo = 0, hi = n_pairs;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (pair_key[mid] < pk)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo >= n_pairs || pair_key[lo] != pk) {
            atomicOr(bad, 16);
            unp_src[e] = 0;
            j1key[e] = SENT;
            continue;
        }
        int64_t b = node_ptr[lo], len = node_ptr[lo + 1] - b;
        int64_t pos = lower_bound_i32(node_idx + b, len, j);
        if (pos >= len || node_idx[b + pos] != j) atomicOr(bad, 16);
        // the piece of the pair holding position pos: the last one starting at
        // or before it
        int64_t a = pair_piece[lo], z = pair_piece[lo + 1] - 1;
        if (z < a) {
            atomicOr(bad, 16);
            unp_src[e] = 0;
            j1key[e] = SENT;
            continue;
        }
        while (a < z) {
            int64_t mid = (a + z + 1) >> 1;
            if (piece_lo[mid] <= pos)
                a = mid;
            else
                z = mid - 1;
        }
        int64_t q = piece_dst[a];
        j1key[e] = ((int64_t)t != q) ? (((uint64_t)q << (rb + jb)) | (t << jb) | (uint64_t)j)
                                     : SENT;
        unp_src[e] = (int32_t)(piece_gr[a] + pos - piece_lo[a]);
    }
}

// Three-block CSR: every row's entries reordered on_process | on_node |
// off_node (stored order kept inside a block), columns coded by block.
__global__ void k_three_block(const int64_t *rp, int64_t n, const int32_t *col, const double *val,
                              const uint8_t *tag, Part part, const int32_t *bll_ptr,
                              const int32_t *bll_j, const int32_t *bnl_ptr, const int32_t *bnl_j,
                              uint32_t *colenc, double *val_out, float *val32_out,
                              int32_t *split, int32_t *rowptr32, int *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = part.owner(i);
        int64_t pos = rp[i];
        rowptr32[i] = (int32_t)rp[i];
        if (i == n - 1) rowptr32[n] = (int32_t)rp[n];
        for (int blk = 0; blk < 3; blk++) {
            int32_t cnt = 0;
            for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
                if (tag[k] != blk) continue;
                int32_t j = col[k];
                uint32_t enc;
                if (blk == 0) {
                    enc = (uint32_t)j;
                } else {
                    const int32_t *ptr = blk == 1 ? bll_ptr : bnl_ptr;
                    const int32_t *arr = blk == 1 ? bll_j : bnl_j;
                    int64_t b = ptr[t], len = ptr[t + 1] - b;
                    int64_t p = lower_bound_i32(arr + b, len, j);
                    if (p >= len || arr[b + p] != j) atomicOr(bad, 32);
                    enc = ((uint32_t)blk << kBlockShift) | (uint32_t)(b + p);
                }
                colenc[pos] = enc;
                val_out[pos] = val[k];
                if (val32_out) val32_out[pos] = (float)val[k];
                pos++;
                cnt++;
            }
            split[3 * i + blk] = cnt;
        }
    }
}

// Lengths of every row's on_process part (L) and remote part (R); the entry
// after the last row is 0 so that an exclusive scan ends with the totals.
__global__ void k_split_lens(const int32_t *split, int64_t n, int32_t *lenL, int32_t *lenR)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x) {
        lenL[i] = i < n ? split[3 * i] : 0;
        lenR[i] = i < n ? split[3 * i + 1] + split[3 * i + 2] : 0;
    }
}

// Copies each three-block row into its L part (the first split[3i] entries)
// and R part (the rest), keeping the order.
__global__ void k_split_copy(const int32_t *rp, int64_t n, const uint32_t *col, const double *val,
                             const float *val32, const int32_t *rpL, const int32_t *rpR,
                             uint32_t *colL, double *valL, float *val32L, uint32_t *colR,
                             double *valR, float *val32R)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = rp[i], nl = rpL[i + 1] - rpL[i], e = rp[i + 1];
        for (int32_t k = 0; k < nl; k++) {
            colL[rpL[i] + k] = col[b + k];
            valL[rpL[i] + k] = val[b + k];
            if (val32L) val32L[rpL[i] + k] = val32[b + k];
        }
        for (int32_t k = b + nl; k < e; k++) {
            const int32_t q = rpR[i] + (k - b - nl);
            colR[q] = col[k];
            valR[q] = val[k];
            if (val32R) val32R[q] = val32[k];
        }
    }
}

// ------------------------------------------------------------ CUB helpers

struct Cub {
    cudaStream_t st = 0;
    dvec<char> tmp;
    dvec<int> num;
    Cub() : num(1) {}
    void *temp(size_t bytes)
    {
        if ((int64_t)bytes > tmp.n) tmp.alloc((int64_t)bytes + 256);
        return tmp.p;
    }
    int64_t read_num()
    {
        int h = 0;
        CK(cudaMemcpy(&h, num.p, sizeof(int), cudaMemcpyDeviceToHost));
        return h;
    }
    template <class F>
    int64_t select(const uint64_t *in, int64_t n, uint64_t *out, F f)
    {
        if (n == 0) return 0;
        size_t b = 0;
        CK(cub::DeviceSelect::If(nullptr, b, in, out, num.p, (int)n, f, st));
        CK(cub::DeviceSelect::If(temp(b), b, in, out, num.p, (int)n, f, st));
        return read_num();
    }
    // sorts keys[0..n) ascending over bits [0, end_bit); alt is scratch
    void sort(uint64_t *keys, uint64_t *alt, int64_t n, int end_bit)
    {
        if (n <= 1) return;
        cub::DoubleBuffer<uint64_t> db(keys, alt);
        size_t b = 0;
        CK(cub::DeviceRadixSort::SortKeys(nullptr, b, db, (int)n, 0, end_bit, st));
        CK(cub::DeviceRadixSort::SortKeys(temp(b), b, db, (int)n, 0, end_bit, st));
        if (db.Current() != keys)
            CK(cudaMemcpyAsync(keys, db.Current(), sizeof(uint64_t) * n,
                               cudaMemcpyDeviceToDevice, st));
    }
    int64_t unique(const uint64_t *in, int64_t n, uint64_t *out)
    {
        if (n == 0) return 0;
        size_t b = 0;
        CK(cub::DeviceSelect::Unique(nullptr, b, in, out, num.p, (int)n, st));
        CK(cub::DeviceSelect::Unique(temp(b), b, in, out, num.p, (int)n, st));
        return read_num();
    }
    // runs of equal keys: unique values and lengths, copied to the host
    void rle(const uint64_t *in, int64_t n, std::vector<uint64_t> &uniq,
             std::vector<int32_t> &len)
    {
        uniq.clear();
        len.clear();
        if (n == 0) return;
        dvec<uint64_t> u(n);
        dvec<int32_t> c(n);
        size_t b = 0;
        CK(cub::DeviceRunLengthEncode::Encode(nullptr, b, in, u.p, c.p, num.p, (int)n, st));
        CK(cub::DeviceRunLengthEncode::Encode(temp(b), b, in, u.p, c.p, num.p, (int)n, st));
        int64_t m = read_num();
        uniq.resize(m);
        len.resize(m);
        CK(cudaMemcpy(uniq.data(), u.p, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(len.data(), c.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    }
};

// Sliced rows: one warp per chunk copies each lane's row into the chunk's
// column-major slots (slot first + i * lanes + lane holds entry i of the
// lane's row) and pads the slots past the row's end.
__global__ void k_sell_fill(const int32_t *rp, const uint32_t *col, const double *val,
                            const float *val32, const int2 *info, const int32_t *perm,
                            int64_t nch, uint32_t *scol, double *sval, float *sval32)
{
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= nch) return;
    const int2 inf = info[c];
    const int width = inf.y >> 6, nl = inf.y & 63;
    if (lane >= nl) return;
    const int row = perm[32 * c + lane];
    const int k0 = rp[row], len = rp[row + 1] - k0;
    for (int i = 0; i < width; i++) {
        const int64_t q = (int64_t)inf.x + (int64_t)i * nl + lane;
        const bool in = i < len;
        scol[q] = in ? col[k0 + i] : kSellPad;
        sval[q] = in ? val[k0 + i] : 0.0;
        if (sval32) sval32[q] = in ? val32[k0 + i] : 0.0f;
    }
}

// A sorted, unique key array (prefix << jb | j) becomes a message list whose
// prefix is (src << fb | dst); with fb < 0 the prefix is one process id used
// as both src and dst (the per-process buffer layouts).
// Majority mapping (the alternative named after Eq. U), sending side: for
// node pair k (messages of the NODE list, ascending (src, dst)), how many
// values of E(n,m) each process of n owns.  cnt: [M][ppn].
__global__ void k_major_send(const int32_t *idx, int64_t total, const int64_t *ptr, int64_t M,
                             const int32_t *src_node, Part part, int32_t ppn, int32_t *cnt)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = M - 1;  // the pair k with ptr[k] <= e < ptr[k + 1]
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (ptr[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const int64_t p = part.owner(idx[e]) - (int64_t)src_node[lo] * ppn;
        atomicAdd(&cnt[lo * ppn + p], 1);
    }
}
// Receiving side: every (t, j) of the off-node receive sets (key t << jb | j)
// is a value of E(owner(j)'s node, t's node) that process t's rows use.
__global__ void k_major_recv(const uint64_t *tj, int64_t n, int jb, const uint64_t *pair_key,
                             int64_t M, int nb, Part part, int32_t ppn, int32_t *cnt, int *bad)
{
    const uint64_t jmask = (1ull << jb) - 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (int64_t)(tj[e] >> jb), j = (int64_t)(tj[e] & jmask);
        const int64_t sn = part.owner(j) / ppn, dn = t / ppn;
        const uint64_t key = ((uint64_t)sn << nb) | (uint64_t)dn;
        int64_t lo = 0, hi = M - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (pair_key[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        if (M == 0 || pair_key[lo] != key) {
            atomicOr(bad, 64);
            continue;
        }
        atomicAdd(&cnt[lo * ppn + (t - dn * ppn)], 1);
    }
}

void make_list(Cub &cb, const uint64_t *keys, int64_t cnt, int fb, int jb, HostList &L)
{
    L = HostList();
    L.ptr.assign(1, 0);
    if (cnt == 0) return;
    dvec<uint64_t> pre(cnt);
    k_shift<<<blocks_for(cnt), 256, 0, cb.st>>>(keys, cnt, jb, pre.p);
    CK(cudaGetLastError());
    std::vector<uint64_t> u;
    std::vector<int32_t> len;
    cb.rle(pre.p, cnt, u, len);
    L.m = (int64_t)u.size();
    L.total = cnt;
    L.src.resize(L.m);
    L.dst.resize(L.m);
    L.ptr.resize(L.m + 1);
    L.ptr[0] = 0;
    for (int64_t k = 0; k < L.m; k++) {
        if (fb < 0) {
            L.src[k] = L.dst[k] = (int32_t)u[k];
        } else {
            L.src[k] = (int32_t)(u[k] >> fb);
            L.dst[k] = (int32_t)(u[k] & ((1ull << fb) - 1));
        }
        L.ptr[k + 1] = L.ptr[k] + len[k];
    }
    CK(cudaMalloc(&L.d_idx, sizeof(int32_t) * cnt));
    k_low<<<blocks_for(cnt), 256, 0, cb.st>>>(keys, cnt, (1ull << jb) - 1, L.d_idx);
    CK(cudaGetLastError());
}

// Per-process offsets [np+1] of a per-process layout list (empty ranks too).
std::vector<int32_t> full_ptr(const HostList &L, int32_t np)
{
    std::vector<int32_t> p(np + 1, 0);
    std::vector<int64_t> cnt(np, 0);
    for (int64_t k = 0; k < L.m; k++) cnt[L.src[k]] = L.ptr[k + 1] - L.ptr[k];
    for (int32_t r = 0; r < np; r++) p[r + 1] = (int32_t)(p[r] + cnt[r]);
    return p;
}

int check_bad(const dvec<int> &bad, const char *what)
{
    int h = 0;
    CK(cudaMemcpy(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) throw NapError{NAPSPMV_ERR_ARG, std::string(what)};
    return 0;
}

void host_stats(napspmv_plan_t *P)
{
    napspmv_stats &S = P->stats;
    int64_t np = P->np, ppn = P->ppn;
    std::vector<int64_t> a(4 * np, 0), b(4 * np, 0);
    const HostList &St = P->lists[L_STD];
    for (int64_t k = 0; k < St.m; k++) {
        int64_t len = St.ptr[k + 1] - St.ptr[k];
        bool inter = (St.src[k] / ppn) != (St.dst[k] / ppn);
        S.std_msgs++;
        S.std_vals += len;
        if (inter) {
            S.std_inter_msgs++;
            S.std_inter_vals += len;
            a[4 * St.src[k] + 0]++;
            a[4 * St.src[k] + 1] += len;
        } else {
            S.std_intra_msgs++;
            S.std_intra_vals += len;
            a[4 * St.src[k] + 2]++;
            a[4 * St.src[k] + 3] += len;
        }
        S.std_max_msg_vals = std::max(S.std_max_msg_vals, len);
    }
    const HostList &In = P->lists[L_INTER];
    for (int64_t k = 0; k < In.m; k++) {
        int64_t len = In.ptr[k + 1] - In.ptr[k];
        S.nap_inter_msgs++;
        S.nap_inter_vals += len;
        S.nap_max_inter_msg_vals = std::max(S.nap_max_inter_msg_vals, len);
        b[4 * In.src[k] + 0]++;
        b[4 * In.src[k] + 1] += len;
    }
    int64_t *jm[3] = {&S.j0_msgs, &S.j1_msgs, &S.j2_msgs};
    int64_t *jv[3] = {&S.j0_vals, &S.j1_vals, &S.j2_vals};
    const int lk[3] = {L_J0, L_J1, L_J2};
    for (int q = 0; q < 3; q++) {
        const HostList &J = P->lists[lk[q]];
        for (int64_t k = 0; k < J.m; k++) {
            int64_t len = J.ptr[k + 1] - J.ptr[k];
            (*jm[q])++;
            (*jv[q]) += len;
            b[4 * J.src[k] + 2]++;
            b[4 * J.src[k] + 3] += len;
        }
    }
    S.nap_intra_msgs = S.j0_msgs + S.j1_msgs + S.j2_msgs;
    S.nap_intra_vals = S.j0_vals + S.j1_vals + S.j2_vals;
    for (int64_t r = 0; r < np; r++) {
        S.std_max_inter_msgs_proc = std::max(S.std_max_inter_msgs_proc, a[4 * r + 0]);
        S.std_max_inter_vals_proc = std::max(S.std_max_inter_vals_proc, a[4 * r + 1]);
        S.std_max_intra_msgs_proc = std::max(S.std_max_intra_msgs_proc, a[4 * r + 2]);
        S.std_max_intra_vals_proc = std::max(S.std_max_intra_vals_proc, a[4 * r + 3]);
        S.nap_max_inter_msgs_proc = std::max(S.nap_max_inter_msgs_proc, b[4 * r + 0]);
        S.nap_max_inter_vals_proc = std::max(S.nap_max_inter_vals_proc, b[4 * r + 1]);
        S.nap_max_intra_msgs_proc = std::max(S.nap_max_intra_msgs_proc, b[4 * r + 2]);
        S.nap_max_intra_vals_proc = std::max(S.nap_max_intra_vals_proc, b[4 * r + 3]);
    }
    S.node_pairs = P->lists[L_NODE].m;
    S.bll_total = P->n_bll;
    S.bnl_total = P->n_bnl;
    S.lbuf_total = P->n_lbuf;
    double N = (double)P->n, nnz = (double)P->nnz;
    S.bytes_csr_f64 = 4.0 * (N + 1) + nnz * 12.0 + 16.0 * N;
    S.bytes_csr_f32 = 4.0 * (N + 1) + nnz * 8.0 + 16.0 * N;
    S.bytes_msg = 20.0 * (double)(P->n_bll + P->n_lbuf + P->n_gs + P->n_bnl) + 20.0 * (double)P->n_gs;
}

// Sliced-row copy of one matrix part (which: 0 whole, 1 local, 2 remote) from
// its CSR (host row pointer hrp, device arrays).  Windows: the rows of each
// process (contiguous partition) or of each 1024-row block (strided).  Within
// a window, rows of at most kSellLong entries are sorted by count, longest
// first (ties by row), and cut into chunks of up to 32 whose counts are at
// least half the first one's; longer rows are listed apart.  A part whose
// padded slots would not fit 31-bit offsets is left without a sliced copy.
void build_sell(napspmv_plan_t *P, int which, const std::vector<int32_t> &hrp,
                const int32_t *d_rp, const uint32_t *d_col, const double *d_val,
                const float *d_val32, const Part &part)
{
    SellPart &S = P->sell[which];
    const int64_t n = P->n;
    std::vector<int2> info;
    std::vector<int32_t> perm, lrows, ord;
    int64_t slots = 0;
    auto len = [&](int32_t r) { return hrp[r + 1] - hrp[r]; };
    auto window = [&](int64_t r0, int64_t r1) {
        ord.clear();
        for (int64_t r = r0; r < r1; r++) {
            if (len((int32_t)r) > kSellLong) lrows.push_back((int32_t)r);
            else ord.push_back((int32_t)r);
        }
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int32_t a, int32_t b) { return len(a) > len(b); });
        size_t j = 0;
        while (j < ord.size()) {
            const int32_t w = len(ord[j]);
            size_t e = j + 1;
            while (e < ord.size() && e - j < 32 && 2 * len(ord[e]) >= w) e++;
            const int nl = (int)(e - j);
            info.push_back(make_int2((int)std::min<int64_t>(slots, INT32_MAX), (w << 6) | nl));
            for (int l = 0; l < 32; l++) perm.push_back(l < nl ? ord[j + l] : -1);
            // every chunk starts on a 4-slot (16-byte) boundary: its column
            // blocks are copied into shared memory with bulk copies
            slots += ((int64_t)w * nl + 3) & ~3ll;
            j = e;
        }
    };
    if (part.strided) {
        for (int64_t r0 = 0; r0 < n; r0 += 1024) window(r0, std::min<int64_t>(n, r0 + 1024));
    } else {
        for (int64_t r = 0; r < part.np; r++) window(part.start(r), part.start(r + 1));
    }
    if (slots > (int64_t)INT32_MAX - 1024) {
        S.slots = -1;  // no sliced copy: NAPSPMV_PIPELINE_SELL is refused for this plan
        return;
    }
    S.nch = (int64_t)info.size();
    S.slots = slots;
    S.n_long = (int32_t)lrows.size();
    S.d_info = upload(info);
    S.d_perm = upload(perm);
    S.d_long = upload(lrows);
    // padded past the last slot: a block's bulk copy is widened to 16 bytes
    auto al = [&](size_t sz) {
        void *q = nullptr;
        CK(cudaMalloc(&q, sz * (size_t)std::max<int64_t>(slots, 1) + 256));
        CK(cudaMemset(q, 0, sz * (size_t)std::max<int64_t>(slots, 1) + 256));
        return q;
    };
    S.d_col = (uint32_t *)al(4);
    S.d_val = (double *)al(8);
    if (d_val32) S.d_val32 = (float *)al(4);
    if (S.nch) {
        k_sell_fill<<<blocks_for(32 * S.nch), 256>>>(d_rp, d_col, d_val, d_val32, S.d_info,
                                                     S.d_perm, S.nch, S.d_col, S.d_val,
                                                     S.d_val32);
        CK(cudaGetLastError());
    }
}

void build(napspmv_plan_t *P, const napspmv_csr *A)
{
    const int64_t n = A->n, nnz = A->nnz;
    const int32_t np = P->np, ppn = P->ppn, nn = P->nn;
    Cub cb;
    Part part{n / np, n % np, (n % np) * (n / np + 1), np,
              (P->flags & NAPSPMV_PARTITION_STRIDED) != 0};
    const int jb = bits_for(n - 1), rb = bits_for(np - 1), nb = bits_for(nn - 1);
    if (2 * rb + jb > 63)
        throw NapError{NAPSPMV_ERR_UNSUPPORTED, "N and n_p too large for 64-bit plan keys"};

    // ---- upload and validate the CSR
    dvec<int64_t> rp(n + 1);
    dvec<int32_t> col(nnz);
    dvec<double> val(nnz);
    CK(cudaMemcpy(rp.p, A->row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault));
    if (nnz) {
        CK(cudaMemcpy(col.p, A->col, sizeof(int32_t) * nnz, cudaMemcpyDefault));
        CK(cudaMemcpy(val.p, A->val, sizeof(double) * nnz, cudaMemcpyDefault));
    }
    dvec<int> bad(1);
    CK(cudaMemset(bad.p, 0, sizeof(int)));
    k_check_rowptr<<<blocks_for(n), 256>>>(rp.p, n, nnz, bad.p);
    CK(cudaGetLastError());
    check_bad(bad, "row_ptr must start at 0, never decrease and end at nnz");
    dvec<int32_t> row_of(nnz);
    k_row_of<<<blocks_for(n), 256>>>(rp.p, n, col.p, row_of.p, bad.p);
    CK(cudaGetLastError());
    check_bad(bad, "column index out of range [0, n)");

    dvec<uint64_t> keys(nnz), alt(nnz);
    if (nnz) {
        k_pair_keys<<<blocks_for(nnz), 256>>>(row_of.p, col.p, nnz, jb, keys.p);
        CK(cudaGetLastError());
        cb.sort(keys.p, alt.p, nnz, 2 * jb);
        k_adjacent_equal<<<blocks_for(nnz), 256>>>(keys.p, nnz, bad.p);
        CK(cudaGetLastError());
        check_bad(bad, "an entry (i, j) is stored twice");
    }

    // ---- classify; the standard plan (Eqs. P, D)
    dvec<uint8_t> tag(nnz);
    dvec<unsigned long long> blk(3);
    CK(cudaMemset(blk.p, 0, 3 * sizeof(unsigned long long)));
    if (nnz) {
        k_classify<<<blocks_for(nnz), 256>>>(row_of.p, col.p, nnz, part, ppn, rb, jb, tag.p,
                                             keys.p, blk.p);
        CK(cudaGetLastError());
    }
    unsigned long long hb[3];
    CK(cudaMemcpy(hb, blk.p, sizeof(hb), cudaMemcpyDeviceToHost));
    P->stats.nnz_on_process = (int64_t)hb[0];
    P->stats.nnz_on_node = (int64_t)hb[1];
    P->stats.nnz_off_node = (int64_t)hb[2];
    row_of.alloc(0);

    int64_t c = cb.select(keys.p, nnz, alt.p, NotSent{});
    cb.sort(alt.p, keys.p, c, 2 * rb + jb);
    dvec<uint64_t> std_u(c);
    int64_t U = cb.unique(alt.p, c, std_u.p);
    make_list(cb, std_u.p, U, rb, jb, P->lists[L_STD]);

    // on-node part: J2 (Eqs. L2, IL2) and b_{l->l}; off-node part: E, b_{nl->l}
    dvec<uint64_t> on_u(U), off_u(U);
    int64_t n_on = cb.select(std_u.p, U, on_u.p, SameNode{rb, jb, ppn, true});
    int64_t n_off = cb.select(std_u.p, U, off_u.p, SameNode{rb, jb, ppn, false});
    std_u.alloc(0);
    make_list(cb, on_u.p, n_on, rb, jb, P->lists[L_J2]);

    dvec<uint64_t> tj(std::max(n_on, n_off)), tj_alt(std::max(n_on, n_off));
    if (n_on) {
        k_rekey_tj<<<blocks_for(n_on), 256>>>(on_u.p, n_on, rb, jb, tj.p);
        CK(cudaGetLastError());
    }
    cb.sort(tj.p, tj_alt.p, n_on, rb + jb);
    make_list(cb, tj.p, n_on, -1, jb, P->lists[L_BLL]);
    on_u.alloc(0);

    if (n_off) {
        k_rekey_tj<<<blocks_for(n_off), 256>>>(off_u.p, n_off, rb, jb, tj.p);
        CK(cudaGetLastError());
    }
    cb.sort(tj.p, tj_alt.p, n_off, rb + jb);
    dvec<uint64_t> bnl_keys(n_off);
    if (n_off)
        CK(cudaMemcpy(bnl_keys.p, tj.p, sizeof(uint64_t) * n_off, cudaMemcpyDeviceToDevice));
    make_list(cb, tj.p, n_off, -1, jb, P->lists[L_BNL]);

    // node plan (Eqs. N, E)
    if (n_off) {
        k_rekey_node<<<blocks_for(n_off), 256>>>(off_u.p, n_off, rb, jb, nb, ppn, tj.p);
        CK(cudaGetLastError());
    }
    cb.sort(tj.p, tj_alt.p, n_off, 2 * nb + jb);
    dvec<uint64_t> node_u(n_off);
    int64_t n_node = cb.unique(tj.p, n_off, node_u.p);
    make_list(cb, node_u.p, n_node, nb, jb, P->lists[L_NODE]);
    off_u.alloc(0);
    tj.alloc(0);
    tj_alt.alloc(0);

    P->n_bll = P->lists[L_BLL].total;
    P->n_bnl = P->lists[L_BNL].total;
    if (P->n_bll >= (1ll << 30) || P->n_bnl >= (1ll << 30))
        throw NapError{NAPSPMV_ERR_UNSUPPORTED, "receive buffer beyond 2^30 values"};

    // ---- T, U (host; O(node pairs))
    const HostList &ND = P->lists[L_NODE];
    const int64_t M = ND.m;
    P->send_proc.assign(M, 0);
    P->recv_proc.assign(M, 0);
    // processes per pair on each side: 1, or a group when the node is split
    std::vector<int32_t> send_cnt(M, 1), recv_cnt(M, 1);
    {
        auto procs = [&](int64_t node) { return (int64_t)std::min<int64_t>(ppn, np - node * ppn); };
        std::vector<std::vector<int64_t>> out_of(nn), in_of(nn);
        for (int64_t k = 0; k < M; k++) {
            out_of[ND.src[k]].push_back(k);
            in_of[ND.dst[k]].push_back(k);
        }
        auto len = [&](int64_t k) { return ND.ptr[k + 1] - ND.ptr[k]; };
        const bool majority = (P->flags & NAPSPMV_MAP_MAJORITY) != 0;
        if (majority && M > 0) {
            // per pair: the process of n owning the most of E(n,m) sends, the
            // process of m whose rows use the most of it receives (ties: lowest)
            dvec<int32_t> cs(M * ppn), cr(M * ppn);
            CK(cudaMemset(cs.p, 0, sizeof(int32_t) * M * ppn));
            CK(cudaMemset(cr.p, 0, sizeof(int32_t) * M * ppn));
            std::vector<uint64_t> pk(M);
            for (int64_t k = 0; k < M; k++) pk[k] = ((uint64_t)ND.src[k] << nb) | (uint64_t)ND.dst[k];
            dvec<int64_t> d_ptr;
            d_ptr.p = upload(ND.ptr);
            dvec<int32_t> d_src;
            d_src.p = upload(ND.src);
            dvec<uint64_t> d_pk;
            d_pk.p = upload(pk);
            k_major_send<<<blocks_for(ND.total), 256>>>(ND.d_idx, ND.total, d_ptr.p, M, d_src.p,
                                                       part, ppn, cs.p);
            CK(cudaGetLastError());
            if (P->n_bnl > 0) {
                k_major_recv<<<blocks_for(P->n_bnl), 256>>>(bnl_keys.p, P->n_bnl, jb, d_pk.p, M, nb,
                                                           part, ppn, cr.p, bad.p);
                CK(cudaGetLastError());
            }
            check_bad(bad, "internal: off-node receive value without a node pair");
            std::vector<int32_t> hs(M * ppn), hr(M * ppn);
            CK(cudaMemcpy(hs.data(), cs.p, sizeof(int32_t) * M * ppn, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(hr.data(), cr.p, sizeof(int32_t) * M * ppn, cudaMemcpyDeviceToHost));
            for (int64_t k = 0; k < M; k++) {
                int64_t bs = 0, br = 0;
                for (int64_t p = 1; p < procs(ND.src[k]); p++)
                    if (hs[k * ppn + p] > hs[k * ppn + bs]) bs = p;
                for (int64_t p = 1; p < procs(ND.dst[k]); p++)
                    if (hr[k * ppn + p] > hr[k * ppn + br]) br = p;
                P->send_proc[k] = (int32_t)bs;
                P->recv_proc[k] = (int32_t)br;
            }
        }
        for (int64_t x = 0; x < (majority ? 0 : nn); x++) {
            auto &o = out_of[x];
            std::stable_sort(o.begin(), o.end(), [&](int64_t a, int64_t b) {
                if (len(a) != len(b)) return len(a) > len(b);
                return ND.dst[a] < ND.dst[b];
            });
            const int64_t px = procs(x);
            const bool split = (P->flags & NAPSPMV_MAP_SPLIT) != 0;
            // node splitting (the text after Eq. U): fewer partners than
            // processes -> partner k gets px / K (+1 for the first px mod K)
            // consecutive processes, counted up from process 0 when sending
            if (split && (int64_t)o.size() < px) {
                const int64_t K = (int64_t)o.size();
                int64_t first = 0;
                for (int64_t k = 0; k < K; k++) {
                    const int64_t size = px / K + (k < px % K ? 1 : 0);
                    P->send_proc[o[k]] = (int32_t)first;
                    send_cnt[o[k]] = (int32_t)size;
                    first += size;
                }
            } else {
                for (size_t k = 0; k < o.size(); k++) P->send_proc[o[k]] = (int32_t)(k % px);
            }
            auto &i = in_of[x];
            bool text = (P->flags & NAPSPMV_MAP_TEXT) != 0;
            std::stable_sort(i.begin(), i.end(), [&](int64_t a, int64_t b) {
                if (len(a) != len(b)) return text ? len(a) > len(b) : len(a) < len(b);
                return ND.src[a] < ND.src[b];
            });
            // receiving: groups counted down from the last process
            if (split && (int64_t)i.size() < px) {
                const int64_t K = (int64_t)i.size();
                int64_t top = px;
                for (int64_t k = 0; k < K; k++) {
                    const int64_t size = px / K + (k < px % K ? 1 : 0);
                    P->recv_proc[i[k]] = (int32_t)(top - size);
                    recv_cnt[i[k]] = (int32_t)size;
                    top -= size;
                }
            } else {
                for (size_t k = 0; k < i.size(); k++)
                    P->recv_proc[i[k]] = (int32_t)(px - 1 - (int64_t)(k % px));
            }
        }
    }

    // ---- G, I: one message per node pair, in (src, dst) order for g_send and
    // (dst, src) order for g_recv.  With node splitting a pair carries
    // c = max(send group, receive group) messages: piece i of E(n,m) (positions
    // floor(i e / c) .. floor((i + 1) e / c) - 1) from the i-th process of the
    // sending group to the i-th of the receiving group, cyclically; empty
    // pieces are no message.
    struct Msg {
        int32_t pair, src, dst;
        int64_t lo, hi;  // positions in E(n,m)
    };
    std::vector<Msg> msgs;
    msgs.reserve(M);
    std::vector<int64_t> pair_piece(M + 1, 0);  // first message (by pair) of each pair
    for (int64_t k = 0; k < M; k++) {
        const int64_t ns = send_cnt[k], nr = recv_cnt[k], c = std::max(ns, nr);
        const int64_t e = ND.ptr[k + 1] - ND.ptr[k];
        for (int64_t i = 0; i < c; i++) {
            const int64_t lo = i * e / c, hi = (i + 1) * e / c;
            if (hi == lo) continue;
            Msg mg;
            mg.pair = (int32_t)k;
            mg.src = (int32_t)(ND.src[k] * ppn + P->send_proc[k] + i % ns);
            mg.dst = (int32_t)(ND.dst[k] * ppn + P->recv_proc[k] + i % nr);
            mg.lo = lo;
            mg.hi = hi;
            msgs.push_back(mg);
        }
        pair_piece[k + 1] = (int64_t)msgs.size();
    }
    const int64_t NM = (int64_t)msgs.size();
    std::vector<int32_t> sorder(NM), rorder(NM);
    std::iota(sorder.begin(), sorder.end(), 0);
    std::iota(rorder.begin(), rorder.end(), 0);
    std::sort(sorder.begin(), sorder.end(), [&](int32_t a, int32_t b) {
        return msgs[a].src != msgs[b].src ? msgs[a].src < msgs[b].src : msgs[a].dst < msgs[b].dst;
    });
    std::sort(rorder.begin(), rorder.end(), [&](int32_t a, int32_t b) {
        return msgs[a].dst != msgs[b].dst ? msgs[a].dst < msgs[b].dst : msgs[a].src < msgs[b].src;
    });
    // g_recv offset of every message (indexed by message in pair order)
    std::vector<int64_t> gr_off(NM, 0);
    {
        int64_t o = 0;
        for (int64_t i = 0; i < NM; i++) {
            gr_off[rorder[i]] = o;
            o += msgs[rorder[i]].hi - msgs[rorder[i]].lo;
        }
    }
    // g_send in (src, dst) order: offsets, and per message (in that order) its
    // pair, first position in E(n,m), sender and g_recv offset
    std::vector<int64_t> gs_off(NM + 1, 0), msg_gr(NM), msg_lo(NM);
    std::vector<int32_t> msg_pair(NM), msg_src(NM);
    for (int64_t i = 0; i < NM; i++) {
        const Msg &mg = msgs[sorder[i]];
        gs_off[i + 1] = gs_off[i] + (mg.hi - mg.lo);
        msg_pair[i] = mg.pair;
        msg_src[i] = mg.src;
        msg_gr[i] = gr_off[sorder[i]];
        msg_lo[i] = mg.lo;
    }
    P->n_gs = gs_off[NM];
    if (P->n_gs >= (1ll << 30))
        throw NapError{NAPSPMV_ERR_UNSUPPORTED, "g_send beyond 2^30 values"};
    {
        HostList &In = P->lists[L_INTER];
        In = HostList();
        In.m = NM;
        In.total = P->n_gs;
        In.src.resize(NM);
        In.dst.resize(NM);
        In.ptr = gs_off;
        for (int64_t i = 0; i < NM; i++) {
            In.src[i] = msgs[sorder[i]].src;
            In.dst[i] = msgs[sorder[i]].dst;
        }
    }
    // per pair, its pieces in position order: first position, receiver and
    // g_recv offset (for the off-node receive entries' unpack sources)
    std::vector<int64_t> piece_lo(NM), piece_gr(NM);
    std::vector<int32_t> piece_dst(NM);
    for (int64_t q = 0; q < NM; q++) {
        piece_lo[q] = msgs[q].lo;
        piece_gr[q] = gr_off[q];
        piece_dst[q] = msgs[q].dst;
    }
    std::vector<int32_t> node_ptr32(M + 1);
    for (int64_t k = 0; k <= M; k++) node_ptr32[k] = (int32_t)ND.ptr[k];
    dvec<int64_t> d_gs_off;
    d_gs_off.p = upload(gs_off);
    dvec<int32_t> d_msg_pair, d_msg_src, d_node_ptr;
    d_msg_pair.p = upload(msg_pair);
    d_msg_src.p = upload(msg_src);
    d_node_ptr.p = upload(node_ptr32);
    dvec<int64_t> d_msg_gr, d_msg_lo;
    d_msg_gr.p = upload(msg_gr);
    d_msg_lo.p = upload(msg_lo);

    const int64_t ngs = P->n_gs;
    dvec<int32_t> msg_of(ngs);
    dvec<uint64_t> j0key(ngs), j0alt(ngs);
    if (ngs) {
        CK(cudaMalloc(&P->lists[L_INTER].d_idx, sizeof(int32_t) * ngs));
        CK(cudaMalloc(&P->d_xfer_dst, sizeof(int32_t) * ngs));
        k_fill_gsend<<<blocks_for(ngs), 256>>>(ngs, d_gs_off.p, NM, d_msg_pair.p, d_msg_src.p,
                                              d_msg_gr.p, d_msg_lo.p, d_node_ptr.p, ND.d_idx,
                                              part, rb, jb, P->lists[L_INTER].d_idx,
                                              P->d_xfer_dst, msg_of.p, j0key.p);
        CK(cudaGetLastError());
    }

    // ---- J0 (Eqs. L0, IL0) and the aggregator buffers b_{l->nl}
    int64_t nj0 = cb.select(j0key.p, ngs, j0alt.p, NotSent{});
    cb.sort(j0alt.p, j0key.p, nj0, 2 * rb + jb);
    dvec<uint64_t> j0u(nj0);
    int64_t Uj0 = cb.unique(j0alt.p, nj0, j0u.p);
    make_list(cb, j0u.p, Uj0, rb, jb, P->lists[L_J0]);
    if (Uj0) {
        k_rekey_tj<<<blocks_for(Uj0), 256>>>(j0u.p, Uj0, rb, jb, j0key.p);
        CK(cudaGetLastError());
    }
    cb.sort(j0key.p, j0alt.p, Uj0, rb + jb);
    make_list(cb, j0key.p, Uj0, -1, jb, P->lists[L_LBUF]);
    P->n_lbuf = Uj0;
    j0key.alloc(0);
    j0alt.alloc(0);
    j0u.alloc(0);

    std::vector<int32_t> lbuf_ptr = full_ptr(P->lists[L_LBUF], np);
    std::vector<int32_t> bll_ptr = full_ptr(P->lists[L_BLL], np);
    std::vector<int32_t> bnl_ptr = full_ptr(P->lists[L_BNL], np);
    P->h_bll_rank = bll_ptr;
    P->h_bnl_rank = bnl_ptr;
    P->d_bll_rank = upload(bll_ptr);
    P->d_bnl_rank = upload(bnl_ptr);
    dvec<int32_t> d_lbuf_ptr, d_bll_ptr, d_bnl_ptr;
    d_lbuf_ptr.p = upload(lbuf_ptr);
    d_bll_ptr.p = upload(bll_ptr);
    d_bnl_ptr.p = upload(bnl_ptr);
    if (ngs) {
        CK(cudaMalloc(&P->d_pack_src, sizeof(uint32_t) * ngs));
        k_pack_src<<<blocks_for(ngs), 256>>>(ngs, P->lists[L_INTER].d_idx, msg_of.p, d_msg_src.p,
                                            d_lbuf_ptr.p, P->lists[L_LBUF].d_idx, part,
                                            P->d_pack_src, bad.p);
        CK(cudaGetLastError());
        check_bad(bad, "internal: pack source missing from the aggregator buffer");
    }
    msg_of.alloc(0);

    // ---- J1 (Eqs. L1_send, IL1) and the unpack sources
    const int64_t nbnl = P->n_bnl;
    std::vector<uint64_t> pair_key(M);
    for (int64_t k = 0; k < M; k++) pair_key[k] = ((uint64_t)ND.src[k] << nb) | ND.dst[k];
    dvec<uint64_t> d_pair_key;
    d_pair_key.p = upload(pair_key);
    dvec<int64_t> d_pair_piece, d_piece_lo, d_piece_gr;
    dvec<int32_t> d_piece_dst;
    d_pair_piece.p = upload(pair_piece);
    d_piece_lo.p = upload(piece_lo);
    d_piece_gr.p = upload(piece_gr);
    d_piece_dst.p = upload(piece_dst);
    dvec<uint64_t> j1key(nbnl), j1alt(nbnl);
    if (nbnl) {
        CK(cudaMalloc(&P->d_unp_src, sizeof(int32_t) * nbnl));
        k_unpack_src<<<blocks_for(nbnl), 256>>>(nbnl, bnl_keys.p, jb, part, ppn, nb, M,
                                               d_pair_key.p, d_pair_piece.p, d_piece_lo.p,
                                               d_piece_dst.p, d_piece_gr.p, d_node_ptr.p,
                                               ND.d_idx, rb, j1key.p, P->d_unp_src, bad.p);
        CK(cudaGetLastError());
        check_bad(bad, "internal: off-node column without a node-pair message");
    }
    int64_t nj1 = cb.select(j1key.p, nbnl, j1alt.p, NotSent{});
    cb.sort(j1alt.p, j1key.p, nj1, 2 * rb + jb);
    make_list(cb, j1alt.p, nj1, rb, jb, P->lists[L_J1]);
    j1key.alloc(0);
    j1alt.alloc(0);
    bnl_keys.alloc(0);

    // ---- three-block CSR
    // padded so that 16-byte bulk copies of a row range may read past the end
    CK(cudaMalloc(&P->d_rowptr, sizeof(int32_t) * (n + 16)));
    CK(cudaMemset(P->d_rowptr, 0, sizeof(int32_t) * (n + 16)));
    CK(cudaMalloc(&P->d_colenc, sizeof(uint32_t) * std::max<int64_t>(nnz, 1) + 64));
    CK(cudaMalloc(&P->d_val, sizeof(double) * std::max<int64_t>(nnz, 1) + 64));
    CK(cudaMalloc(&P->d_split, sizeof(int32_t) * 3 * n));
    if (P->flags & NAPSPMV_F32_VALUES)
        CK(cudaMalloc(&P->d_val32, sizeof(float) * std::max<int64_t>(nnz, 1) + 64));
    k_three_block<<<blocks_for(n), 256>>>(rp.p, n, col.p, val.p, tag.p, part, d_bll_ptr.p,
                                         P->lists[L_BLL].d_idx, d_bnl_ptr.p,
                                         P->lists[L_BNL].d_idx, P->d_colenc, P->d_val,
                                         P->d_val32, P->d_split, P->d_rowptr, bad.p);
    CK(cudaGetLastError());
    check_bad(bad, "internal: column missing from its receive buffer");

    // ---- local / remote split
    {
        dvec<int32_t> lenL(n + 1), lenR(n + 1);
        CK(cudaMalloc(&P->d_rowptrL, sizeof(int32_t) * (n + 16)));
        CK(cudaMalloc(&P->d_rowptrR, sizeof(int32_t) * (n + 16)));
        CK(cudaMemset(P->d_rowptrL, 0, sizeof(int32_t) * (n + 16)));
        CK(cudaMemset(P->d_rowptrR, 0, sizeof(int32_t) * (n + 16)));
        k_split_lens<<<blocks_for(n + 1), 256>>>(P->d_split, n, lenL.p, lenR.p);
        CK(cudaGetLastError());
        size_t b = 0;
        CK(cub::DeviceScan::ExclusiveSum(nullptr, b, lenL.p, P->d_rowptrL, (int)(n + 1)));
        void *tmp = cb.temp(b);
        CK(cub::DeviceScan::ExclusiveSum(tmp, b, lenL.p, P->d_rowptrL, (int)(n + 1)));
        CK(cub::DeviceScan::ExclusiveSum(tmp, b, lenR.p, P->d_rowptrR, (int)(n + 1)));
        P->h_rowptrL.resize(n + 1);
        P->h_rowptrR.resize(n + 1);
        CK(cudaMemcpy(P->h_rowptrL.data(), P->d_rowptrL, sizeof(int32_t) * (n + 1),
                      cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(P->h_rowptrR.data(), P->d_rowptrR, sizeof(int32_t) * (n + 1),
                      cudaMemcpyDeviceToHost));
        P->nnzL = P->h_rowptrL[n];
        P->nnzR = P->h_rowptrR[n];
        const bool f32 = P->d_val32 != nullptr;
        auto al = [&](int64_t m, size_t sz) {
            void *q = nullptr;
            CK(cudaMalloc(&q, sz * (size_t)std::max<int64_t>(m, 1) + 64));
            return q;
        };
        P->d_colL = (uint32_t *)al(P->nnzL, 4);
        P->d_valL = (double *)al(P->nnzL, 8);
        P->d_colR = (uint32_t *)al(P->nnzR, 4);
        P->d_valR = (double *)al(P->nnzR, 8);
        if (f32) {
            P->d_val32L = (float *)al(P->nnzL, 4);
            P->d_val32R = (float *)al(P->nnzR, 4);
        }
        k_split_copy<<<blocks_for(n), 256>>>(P->d_rowptr, n, P->d_colenc, P->d_val, P->d_val32,
                                             P->d_rowptrL, P->d_rowptrR, P->d_colL, P->d_valL,
                                             P->d_val32L, P->d_colR, P->d_valR, P->d_val32R);
        CK(cudaGetLastError());
        int lo = 0, hi = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        CK(cudaStreamCreateWithPriority(&P->aux, cudaStreamNonBlocking, lo));
        CK(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    }
    CK(cudaDeviceSynchronize());

    // ---- first row of every node, where the CTA row tiles are cut
    P->node_rows.assign(nn + 1, 0);
    for (int32_t x = 0; x <= nn; x++) {
        int32_t r = std::min<int64_t>((int64_t)x * ppn, np);
        // strided: every node's rows interleave; the row tiles are cut over
        // all rows as one range
        P->node_rows[x] = part.strided ? (x == 0 ? 0 : n) : part.start(r);
    }
    {
        std::vector<int64_t> h(n + 1);
        CK(cudaMemcpy(h.data(), rp.p, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
        P->h_rowptr.resize(n + 1);
        for (int64_t i = 0; i <= n; i++) P->h_rowptr[i] = (int32_t)h[i];
    }
    // sliced-row copies of the whole matrix and of its two split parts
    build_sell(P, 0, P->h_rowptr, P->d_rowptr, P->d_colenc, P->d_val, P->d_val32, part);
    build_sell(P, 1, P->h_rowptrL, P->d_rowptrL, P->d_colL, P->d_valL, P->d_val32L, part);
    build_sell(P, 2, P->h_rowptrR, P->d_rowptrR, P->d_colR, P->d_valR, P->d_val32R, part);
    CK(cudaDeviceSynchronize());

    host_stats(P);
}

}  // namespace

void plan_free(napspmv_plan_t *P)
{
    if (!P) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(P->device);
    if (P->ws) {
        ws_free(P->ws);
        delete P->ws;
    }
    for (auto &g : P->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &L : P->lists)
        if (L.d_idx) cudaFree(L.d_idx);
    void *ptrs[] = {P->d_split, P->d_rowptr, P->d_colenc, P->d_val, P->d_val32, P->d_pack_src,
                    P->d_xfer_dst, P->d_unp_src,
                    P->items.d_items, P->items.d_tilesL, P->items.d_tilesR,
                    P->items.d_wt, P->items.d_wtL, P->items.d_wtR, P->items.d_tilesRH,
                    P->d_rowptrL, P->d_rowptrR, P->d_colL, P->d_colR, P->d_valL, P->d_valR,
                    P->d_val32L, P->d_val32R, P->d_bll_rank, P->d_bnl_rank};
    if (P->aux) cudaStreamDestroy(P->aux);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &S : P->sell) {
        void *sp[] = {S.d_info, S.d_perm, S.d_col, S.d_val, S.d_val32, S.d_long};
        for (void *p : sp)
            if (p) cudaFree(p);
    }
    delete P;
    cudaSetDevice(cur);
}

int plan_create(const napspmv_csr *A, int32_t np, int32_t ppn, uint32_t flags,
                napspmv_plan_t **out)
{
    auto t0 = std::chrono::steady_clock::now();
    if (!out) {
        set_error(NAPSPMV_ERR_ARG, "out is NULL");
        return NAPSPMV_ERR_ARG;
    }
    *out = nullptr;
    if (!A || A->n < 1 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val))) {
        set_error(NAPSPMV_ERR_ARG, "invalid CSR descriptor");
        return NAPSPMV_ERR_ARG;
    }
    if (np < 1 || np > A->n || ppn < 1) {
        set_error(NAPSPMV_ERR_ARG, "need 1 <= n_p <= N and ppn >= 1");
        return NAPSPMV_ERR_ARG;
    }
    if (flags & ~(NAPSPMV_F32_VALUES | NAPSPMV_MAP_TEXT | NAPSPMV_PARTITION_STRIDED |
                  NAPSPMV_MAP_MAJORITY | NAPSPMV_COMPOSED_GATHERS | NAPSPMV_MAP_SPLIT)) {
        set_error(NAPSPMV_ERR_ARG, "unknown plan flag");
        return NAPSPMV_ERR_ARG;
    }
    if ((flags & NAPSPMV_MAP_MAJORITY) && (flags & (NAPSPMV_MAP_TEXT | NAPSPMV_MAP_SPLIT))) {
        set_error(NAPSPMV_ERR_ARG, "NAPSPMV_MAP_MAJORITY excludes NAPSPMV_MAP_TEXT and "
                                   "NAPSPMV_MAP_SPLIT");
        return NAPSPMV_ERR_ARG;
    }
    if (A->n >= (1ll << 30) || A->nnz >= (1ll << 31) - 64) {
        set_error(NAPSPMV_ERR_UNSUPPORTED, "N must be < 2^30 and nnz < 2^31");
        return NAPSPMV_ERR_UNSUPPORTED;
    }
    napspmv_plan_t *P = new napspmv_plan_t();
    P->n = A->n;
    P->nnz = A->nnz;
    P->np = np;
    P->ppn = ppn;
    P->nn = (np + ppn - 1) / ppn;
    P->flags = flags;
    try {
        CK(cudaGetDevice(&P->device));
        CK(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));
        build(P, A);
        P->ws = new napspmv_ws_t();
        int rc = ws_alloc(P, P->ws);
        if (rc) throw NapError{rc, "workspace allocation failed"};
        P->ws->owned_by_plan = true;
        // defaults, measured on GB300 (FP64, per apply):
        //  - rows of more than 12 stored entries on average: the phased engine
        //    with the sliced rows (one lane per row, no shared-memory stage,
        //    chunk groups dealt round robin).  2^23-row banded random workload:
        //    1.71 ms, against 2.18 ms overlapped with sliced rows and 2.00 ms
        //    overlapped with two-lane warp tiles (its SpMV step alone: 0.72 ms
        //    against 1.04 ms);
        //  - shorter rows (the stencils): the overlapped engine with CTA tiles,
        //    one lane per row, 512 rows / 1536 entries (3D 7-point 128^3: 76 us,
        //    against 79 us phased and 89 us overlapped with sliced rows).
        // The lane count and tile shape serve the CTA and warp pipelines when an
        // apply asks for them: one lane per row keeps exactly one FP64 FMA per
        // stored entry (GB300's FP64 pipe is the scarce unit); longer rows take
        // more lanes, with 1024-row / 2048-entry tiles.
        double avg = (double)P->nnz / (double)P->n;
        int vec = avg <= 16 ? 1 : avg <= 32 ? 2 : avg <= 96 ? 4 : avg <= 384 ? 16 : 32;
        int rows = 512 / vec;
        int cap = 1536;
        int ctas = 0;  // occupancy maximum
        const bool sell = P->sell[0].slots >= 0 && avg > 12;
        int pipeline = sell ? NAPSPMV_PIPELINE_SELL : NAPSPMV_PIPELINE_CTA;
        int engine = sell ? NAPSPMV_ENGINE_PHASED : NAPSPMV_ENGINE_OVERLAP;
        if (vec > 1) {
            rows = 1024;
            cap = 2048;
        }
        P->defaults.precision = NAPSPMV_PREC_F64;
        P->defaults.engine = engine;
        P->defaults.vec = vec;
        P->defaults.ctas_per_sm = ctas;
        P->defaults.chunk = 2048;
        P->defaults.tile_rows = rows;
        P->defaults.tile_nnz = cap;
        P->defaults.stages = 2;
        P->defaults.pipeline = pipeline;
        P->defaults.halo = NAPSPMV_HALO_ON;
        P->defaults.timeout_ms = 10000;
        P->defaults.debug_stall = 0;
        rc = build_items(P, P->defaults.tile_rows, P->defaults.tile_nnz);
        if (rc) throw NapError{rc, "row-tile construction failed"};
    } catch (const NapError &e) {
        plan_free(P);
        set_error(e.code, e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        plan_free(P);
        set_error(NAPSPMV_ERR_OOM, "host allocation failed");
        return NAPSPMV_ERR_OOM;
    }
    P->stats.plan_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = P;
    return NAPSPMV_OK;
}

}  // namespace nap
