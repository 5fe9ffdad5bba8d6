// internal.h -- data structures shared by the library's translation units.
//
// A plan holds the three-block CSR, the index arrays of every message step of
// the node-aware algorithm and the work-item list of the fused persistent
// kernel; a workspace holds the receive buffers and dependency counters of one
// in-flight apply.  Nothing here is part of the C ABI (include/napspmv.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/napspmv.h"

namespace nap {

// ------------------------------------------------------------------ errors
void set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);
void count_launch(int64_t n = 1);

#define NAP_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::nap::cuda_error(e_, #call); \
    } while (0)

// ----------------------------------------------------------- column coding
// A column of the three-block CSR stores its block in the top two bits:
// 0 = on-process (index into v), 1 = on-node (index into b_{l->l}),
// 2 = off-node (index into b_{nl->l}); the low 30 bits are the index.
constexpr uint32_t kBlockShift = 30;
constexpr uint32_t kIndexMask = (1u << 30) - 1;
// A pack source with the top bit set reads the aggregator buffer b_{l->nl},
// otherwise v.
constexpr uint32_t kFromLbuf = 0x80000000u;

// ------------------------------------------------- row tiles (CTA and warp)
enum ItemKind : int32_t {
    kSpmv = 5,  // rows [b, e) of the three-block SpMV
};

struct Item {
    int32_t kind;
    int32_t node;    // node of the rows
    int32_t b, e;    // row range
    int32_t msg;     // remote tiles cut at process bounds: the process
    int32_t k0, k1;  // stored-entry range [row_ptr[b], row_ptr[e])
    int32_t pad;
};

struct ItemSet {
    int32_t tile_rows = 0, tile_nnz = 0;
    int32_t n_items = 0;  // CTA tiles of the whole matrix (d_items)
    Item *d_tilesL = nullptr, *d_tilesR = nullptr;  // tiles of the split parts
    int32_t n_tilesL = 0, n_tilesR = 0;
    // remote tiles cut at process boundaries (Item::msg = process), for the
    // remote pass with staged receive buffers
    Item *d_tilesRH = nullptr;
    int32_t n_tilesRH = 0;
    // warp tiles (at most tile_rows / 8 rows, tile_nnz / 8 entries) of the whole
    // matrix and of its two split parts
    Item *d_wt = nullptr, *d_wtL = nullptr, *d_wtR = nullptr;
    int32_t n_wt = 0, n_wtL = 0, n_wtR = 0;
    // largest staged tile (entries, rows) of each list, in the order whole /
    // local / remote CTA tiles, whole / local / remote warp tiles, remote tiles
    // cut per process: a stage is sized to what its list needs, not to tile_nnz
    int32_t fit_nnz[7] = {}, fit_rows[7] = {};
    Item *d_items = nullptr;
};

// --------------------------------------------------------------- plan lists
struct HostList {
    int64_t m = 0, total = 0;
    std::vector<int32_t> src, dst;
    std::vector<int64_t> ptr;
    int32_t *d_idx = nullptr;  // global column indices, device
};

enum ListKind { L_STD = 0, L_NODE, L_INTER, L_J0, L_J1, L_J2, L_BLL, L_BNL, L_LBUF, L_COUNT };

// ------------------------------------------------------- sliced rows (SELL)
// One matrix part (whole, local or remote) in sliced-row form: the rows of
// each process (of each 1024-row block for a strided plan) are sorted by
// stored-entry count, longest first (ties by row), and cut into chunks of up
// to 32 rows whose counts lie within a factor of two of the chunk's first.
// Chunk c stores entry i of its lane l at slot info[c].x + i * lanes + l
// (column-major, so a warp reads consecutive slots); a lane's row shorter
// than the chunk's width is padded with kSellPad columns.  Each row keeps its
// stored entry order, so one lane summing it gives the same bits as the
// one-lane-per-row CSR kernels.  Rows longer than kSellLong entries are listed
// apart and summed by a whole warp from the CSR part.
constexpr uint32_t kSellPad = 0xffffffffu;
constexpr int32_t kSellLong = 256;
struct SellPart {
    int64_t nch = 0, slots = 0;
    int32_t n_long = 0;
    int2 *d_info = nullptr;     // per chunk: first slot, (width << 6) | lanes
    int32_t *d_perm = nullptr;  // 32 per chunk: the row of each lane (-1: none)
    uint32_t *d_col = nullptr;  // block-coded columns, kSellPad in the padding
    double *d_val = nullptr;
    float *d_val32 = nullptr;
    int32_t *d_long = nullptr;  // rows of more than kSellLong entries
};

}  // namespace nap

struct napspmv_ws_s {
    napspmv_plan_t *plan = nullptr;
    int device = 0;
    double *bll = nullptr, *lbuf = nullptr, *gsend = nullptr, *grecv = nullptr, *bnl = nullptr;
    double *xtmp = nullptr;            // chained-apply intermediate vector
    // FP32 mode of the phased engines: FP32 copies of the chain's vectors, and
    // whether the receive buffers hold FP32 copies (their contents are then
    // read as float arrays)
    float *x32[2] = {nullptr, nullptr};
    int buf_f32 = 0;
    double *hv = nullptr, *hw = nullptr;  // staging of napspmv_apply_host
    unsigned long long *ctr = nullptr;  // the fused engine's grid barrier: arrivals, generation
    int *err = nullptr;                 // sticky device status
    bool owned_by_plan = false;
};

struct napspmv_plan_s {
    int device = 0;
    int64_t n = 0, nnz = 0;
    int32_t np = 0, ppn = 0, nn = 0;
    uint32_t flags = 0;
    int num_sms = 0;

    nap::HostList lists[nap::L_COUNT];
    std::vector<int32_t> send_proc, recv_proc;  // per NODE pair
    int32_t *d_split = nullptr;                 // 3 per row

    // three-block CSR
    int32_t *d_rowptr = nullptr;
    uint32_t *d_colenc = nullptr;
    double *d_val = nullptr;
    float *d_val32 = nullptr;

    // the same matrix split in two CSR parts for the overlapped engine: the
    // on_process entries (L, columns index v) and the on_node + off_node
    // entries (R, columns coded by block); each row keeps its stored order
    int64_t nnzL = 0, nnzR = 0;
    int32_t *d_rowptrL = nullptr, *d_rowptrR = nullptr;
    uint32_t *d_colL = nullptr, *d_colR = nullptr;
    double *d_valL = nullptr, *d_valR = nullptr;
    float *d_val32L = nullptr, *d_val32R = nullptr;
    std::vector<int32_t> h_rowptrL, h_rowptrR;
    // per-process offsets of b_{l->l} and b_{nl->l} (np + 1 each), host and device
    std::vector<int32_t> h_bll_rank, h_bnl_rank;
    int32_t *d_bll_rank = nullptr, *d_bnl_rank = nullptr;
    cudaStream_t aux = nullptr;  // low-priority stream of the local SpMV
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

    // sizes of the buffers and index arrays of the message steps
    int64_t n_bll = 0, n_lbuf = 0, n_gs = 0, n_bnl = 0;
    uint32_t *d_pack_src = nullptr;  // [n_gs]
    int32_t *d_xfer_dst = nullptr;   // [n_gs]
    int32_t *d_unp_src = nullptr;    // [n_bnl]
    // BLL / LBUF list idx arrays double as the J2 / J0 gather sources.

    // first row of every node (host), where the CTA row tiles are cut
    std::vector<int64_t> node_rows;  // [nn+1]
    std::vector<int32_t> h_rowptr;         // host copy of the row pointer, for tiling

    // sliced-row copies of the whole matrix, its local part and its remote
    // part (index 0, 1, 2), for NAPSPMV_PIPELINE_SELL; built with the plan
    nap::SellPart sell[3];

    nap::ItemSet items;
    // instantiated CUDA graphs of chained phased applies, newest last
    struct GraphEntry {
        const void *v, *w, *ws;
        int32_t reps, prec, vec, tile_rows, tile_nnz, engine, stages, pipeline, ctas_per_sm, halo;
        double scale;
        cudaGraphExec_t exec;
        int64_t kernels;
    };
    std::vector<GraphEntry> graphs;
    napspmv_opts defaults{};
    napspmv_stats stats{};
    napspmv_ws_t *ws = nullptr;  // the plan's own workspace
};

namespace nap {
int build_items(napspmv_plan_t *P, int32_t tile_rows, int32_t tile_nnz);
int ws_alloc(napspmv_plan_t *P, napspmv_ws_t *ws);
void ws_free(napspmv_ws_t *ws);
void plan_free(napspmv_plan_t *P);
napspmv_opts resolve_opts(const napspmv_plan_t *P, const napspmv_opts *o);
// ERR_ARG / ERR_STATE / ERR_UNSUPPORTED (with the message set) for resolved
// options the plan cannot run, else NAPSPMV_OK
int check_opts(const napspmv_plan_t *P, const napspmv_opts &o);
int apply_batch(int32_t count, napspmv_plan_t *const *plans, napspmv_ws_t *const *ws,
                const double *const *v, double *const *w, const int32_t *reps,
                const double *scale, const napspmv_opts *opts, cudaStream_t s);
}  // namespace nap
