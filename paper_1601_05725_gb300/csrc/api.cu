// api.cu -- the C entry points of include/basker.h: handle, device memory, and
// the order of kernel launches for factor, refactor and solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "basker_internal.h"
#include "round_order.h"
#include "refine_internal.h"
#include "solve_internal.h"
#include "trace.cuh"

struct basker_s {
    basker_options opt;
    bk_plan pl;
    bk_solve_plan sp;
    int device = 0;
    std::vector<std::pair<void *, size_t>> allocs;   // device allocations and their bytes
    bk_dev d{};
    bk_solve_dev sd{};
    // level lists of a full factorization (device)
    std::vector<int32_t *> lv_tasks;
    std::vector<int32_t> lv_ntasks;
    std::vector<size_t> lv_smem;
    std::vector<int32_t *> lv_cols;
    std::vector<int32_t> lv_ncols;
    // separators whose in-node phase runs as one dense elimination, by cluster size
    // ([0]: one block, [1]: BK_DENSE_CLUSTER blocks)
    std::vector<int32_t *> lv_dense[2];
    std::vector<int32_t> lv_ndense[2];
    std::vector<size_t> lv_dsmem[2];
    // redo lists (device buffers of n ints each) and their pinned staging
    int32_t *rd_tasks = nullptr, *rd_c0 = nullptr, *rd_cols = nullptr;
    int32_t *h_stage = nullptr;      // pinned, 3n + ntasks + 16 ints
    bk_status *h_status = nullptr;   // pinned
    int32_t *h_task_fail = nullptr;  // pinned
    int32_t epoch = 0, solve_epoch = 0, refno = 0;
    bool factored = false, ws_dirty = false, schedule_valid = true, order_is_symbolic = true;
    double gp_wall_ms = 0.0;     // wall time of the last complete Algorithm 1 pass (host clock)
    double round_us_per_col = 0.0;   // a refactorization round's wall time per column it processed
    bool sep_dense = false;      // refactorizations recompute every separator densely
    // the repair pass (sep_dense): the tasks it serves (every task without
    // descendants), its dynamic shared memory and its persistent blocks
    int32_t *rp_tasks = nullptr;
    int32_t rp_ntasks = 0, rp_ctas = 0;
    size_t rp_smem = 0;
    // the separators' descendant phase on stored patterns: the columns left to the
    // reach kernel (listed on the device) and the fast kernel's shared memory
    int32_t *df_redo = nullptr;
    std::vector<bk_desc_par> df_par;     // the descendant phase's on-chip sizes per ND level
    // the arena as the symbolic pass left it (natural pivots, symbolic pattern and
    // schedule): a factorization first tries the stored-pattern path from it
    int32_t *sym_Li = nullptr, *sym_Ui = nullptr, *sym_n = nullptr;   // sym_n: 8 arrays of n ints
    int64_t *sym_beg = nullptr;                                       // 4 arrays of n int64
    unsigned long long *sym_pool = nullptr;
    int32_t sym_ver = -1;
    double static_factor_ms = 0.0;   // wall time of the last factorization by that path
    bool static_factor_off = false;  // that path rejected too many natural pivots once: not tried again
    int32_t nrhs_cap = 0;
    double *d_vals = nullptr, *d_b = nullptr, *d_x = nullptr;
    int32_t stage_nrhs = 0;
    basker_info_t info{};
    int64_t device_bytes = 0;
    int32_t launches = 0;
    // kernel timing (options.timing): event pairs recorded on the launch stream
    struct timed { cudaEvent_t a, b; int kind; };
    std::vector<timed> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open_ev = nullptr;
    int open_kind = 0;
    // precision 1: FP64 refinement state, and an FP64 twin handle for the
    // factorizations the FP32 factors cannot serve (built on first need)
    bk_refine_dev rf{};
    double *d_norms = nullptr;       // [0] ||B||_inf, [1] pivot growth
    double *h_norms = nullptr;       // pinned: 2 + 3 * ir_cap
    double *d_vals64 = nullptr;      // the values of the last factorization (A's order)
    double *ir_c = nullptr, *ir_r = nullptr, *ir_z = nullptr, *ir_dz = nullptr, *d_irn = nullptr;
    int32_t ir_cap = 0;
    double bnorm = 0.0;
    bool use64 = false, fp32_valid = false;
    // launch sizes chosen by basker_autotune (0: the occupancy defaults)
    int tune_static = 0, tune_solve = 0, tune_dd = 0;
    basker_t twin = nullptr;
    // options.graphs: the launches that follow every factorization (factors into
    // rows, the solve's leaf order), captured once per arena and replayed
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t g_finish = nullptr;
    int32_t arena_ver = 0, g_finish_ver = -1;
    // the symbolic inputs, kept to build the twin
    std::vector<int32_t> in_colptr, in_rowind, in_P, in_Q, in_bptr, in_ndptr;
    int32_t in_nblocks = 0, in_ndblock = -1, in_ndleaves = 0;
};

namespace {

enum { KT_GATHER = 0, KT_STATIC = 1, KT_LEVELS = 2, KT_GP = 3, KT_DESC = 4, KT_SOLVE = 5, KT_DENSE = 6, KT_SPEC = 7,
       KT_ROWS = 8, KT_REFINE = 9 };

cudaEvent_t take_event(basker_t h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket a launch (or a group of launches of one kind) with events on its stream.
void tbeg(basker_t h, int kind, cudaStream_t s, int nkernels)
{
    h->info.kernel_launches += nkernels;
    h->info.kernel_calls[kind]++;
    if (!h->opt.timing) return;
    h->open_ev = take_event(h);
    h->open_kind = kind;
    cudaEventRecord(h->open_ev, s);
}

void tend(basker_t h, cudaStream_t s)
{
    if (!h->opt.timing || !h->open_ev) return;
    cudaEvent_t b = take_event(h);
    cudaEventRecord(b, s);
    h->pending.push_back({h->open_ev, b, h->open_kind});
    h->open_ev = nullptr;
}

void tflush(basker_t h)
{
    for (auto &t : h->pending) {
        float ms = 0.f;
        cudaEventSynchronize(t.b);
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) h->info.kernel_ms[t.kind] += ms;
        h->pool.push_back(t.a);
        h->pool.push_back(t.b);
    }
    h->pending.clear();
}

template <typename T>
int dalloc(basker_t h, T **p, size_t count, bool zero = false)
{
    *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return BASKER_ERR_OOM;
    }
    h->allocs.emplace_back((void *)*p, bytes);
    h->device_bytes += (int64_t)bytes;
    if (zero && cudaMemset(*p, 0, bytes) != cudaSuccess) return BASKER_ERR_CUDA;
    return BASKER_OK;
}

// Stream capture (options.graphs) and calls that synchronize the whole device
// (cudaDeviceSynchronize, cudaFree) must not overlap between threads: a
// device-wide synchronization invalidates another thread's capture.  Captures are
// short (they record launches, nothing runs), so one process-wide lock suffices.
std::mutex g_capture_mu;

void dfree(basker_t h, void *p)
{
    if (!p) return;
    auto it = std::find_if(h->allocs.begin(), h->allocs.end(), [p](const std::pair<void *, size_t> &a) {
        return a.first == p;
    });
    if (it != h->allocs.end()) {
        h->device_bytes -= (int64_t)it->second;
        h->allocs.erase(it);
    }
    std::lock_guard<std::mutex> lk(g_capture_mu);
    cudaFree(p);
}

cudaError_t device_sync()
{
    std::lock_guard<std::mutex> lk(g_capture_mu);
    return cudaDeviceSynchronize();
}

template <typename T>
int upload(basker_t h, T **p, const std::vector<T> &v)
{
    int s = dalloc(h, p, v.size());
    if (s) return s;
    if (!v.empty() && cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return BASKER_ERR_CUDA;
    return BASKER_OK;
}

#define TRY(x)                      \
    do {                            \
        int s_ = (x);               \
        if (s_ != BASKER_OK) return s_; \
    } while (0)
// the last failing runtime call of this thread: its error code and source line
thread_local int g_cuda_err = 0, g_cuda_line = 0;
#define CU(x)                                  \
    do {                                       \
        const cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess) {               \
            cudaGetLastError();                \
            g_cuda_err = (int)e_;              \
            g_cuda_line = __LINE__;            \
            return BASKER_ERR_CUDA;            \
        }                                      \
    } while (0)

// Persistent blocks of the stored-pattern and column-levels kernels.
int static_blocks(basker_t h) { return h->tune_static > 0 ? h->tune_static : bk_static_blocks(); }

// L/U arrays sized by the current layout (symbolic pattern, slack, growth), each
// followed by its spill pool; per-column region starts and ends.
int alloc_factors(basker_t h)
{
    bk_plan &pl = h->pl;
    dfree(h, h->d.Li); dfree(h, (void *)h->d.Lx); dfree(h, h->d.Ui); dfree(h, (void *)h->d.Ux);
    dfree(h, h->d.Lbeg); dfree(h, h->d.Ubeg); dfree(h, h->d.Lend); dfree(h, h->d.Uend);
    h->d.Li = h->d.Ui = nullptr;
    h->d.Lx = h->d.Ux = nullptr;
    h->d.lpool_end = pl.lcap + pl.lpool;
    h->d.upool_end = pl.ucap + pl.upool;
    h->arena_ver++;                   // captured launches hold the old arrays
    // L's arrays carry 16 bytes of slack: the rounds copy columns in 16-byte
    // pieces from the boundary below a column to the one above its end
    TRY(dalloc(h, &h->d.Li, (size_t)h->d.lpool_end + 4));
    // the factors by rows (for the solve) have the same capacities
    bk_rows &r = h->sd.r;
    dfree(h, r.Lrk); dfree(h, r.Lrx); dfree(h, r.Urk); dfree(h, r.Urx); dfree(h, r.tk); dfree(h, r.tx);
    dfree(h, r.Ls);
    r.Lrk = r.Urk = r.tk = r.Ls = nullptr;
    r.Lrx = r.Urx = r.tx = nullptr;
    TRY(dalloc(h, &r.Lrk, (size_t)h->d.lpool_end));
    TRY(dalloc(h, &r.Lrx, (size_t)h->d.lpool_end));
    TRY(dalloc(h, &r.Urk, (size_t)h->d.upool_end));
    TRY(dalloc(h, &r.Urx, (size_t)h->d.upool_end));
    TRY(dalloc(h, &r.tk, (size_t)std::max(h->d.lpool_end, h->d.upool_end)));
    TRY(dalloc(h, &r.Ls, (size_t)h->d.lpool_end));
    TRY(dalloc(h, &r.tx, (size_t)std::max(h->d.lpool_end, h->d.upool_end)));
    TRY(dalloc(h, &h->d.Lx, (size_t)h->d.lpool_end + 4));
    TRY(dalloc(h, &h->d.Ui, (size_t)h->d.upool_end));
    TRY(dalloc(h, &h->d.Ux, (size_t)h->d.upool_end));
    TRY(upload(h, &h->d.Lbeg, pl.sLbeg));
    TRY(upload(h, &h->d.Ubeg, pl.sUbeg));
    std::vector<int64_t> le(pl.sLbeg.begin() + 1, pl.sLbeg.end()), ue(pl.sUbeg.begin() + 1, pl.sUbeg.end());
    TRY(upload(h, &h->d.Lend, le));
    TRY(upload(h, &h->d.Uend, ue));
    unsigned long long next[2] = {(unsigned long long)pl.lcap, (unsigned long long)pl.ucap};
    CU(cudaMemcpy(h->d.pool, next, sizeof next, cudaMemcpyHostToDevice));
    return BASKER_OK;
}

// the symbolic pattern in the L/U arrays (the static path's first schedule)
int upload_symbolic_pattern(basker_t h)
{
    bk_plan &pl = h->pl;
    if (pl.counts_only) {
        // no pattern or schedule: the first factorization runs the complete pass
        // and computes the schedule of its pattern
        if (!h->d.iorder) TRY(upload(h, (int32_t **)&h->d.iorder, pl.iorder));
        h->order_is_symbolic = false;
        return BASKER_OK;
    }
    std::vector<int32_t> Li((size_t)pl.lcap, 0), Ui((size_t)pl.ucap, 0);
    int64_t l = 0, u = 0;
    for (int32_t c = 0; c < pl.n; c++) {
        for (int32_t k = 0; k < pl.sLcnt[(size_t)c]; k++) Li[(size_t)(pl.sLbeg[(size_t)c] + k)] = pl.sLi[(size_t)l++];
        for (int32_t k = 0; k < pl.sUcnt[(size_t)c]; k++) Ui[(size_t)(pl.sUbeg[(size_t)c] + k)] = pl.sUi[(size_t)u++];
    }
    CU(cudaMemcpy(h->d.Li, Li.data(), Li.size() * 4, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->d.Ui, Ui.data(), Ui.size() * 4, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->d.Lcnt, pl.sLcnt.data(), (size_t)pl.n * 4, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->d.Ucnt, pl.sUcnt.data(), (size_t)pl.n * 4, cudaMemcpyHostToDevice));
    std::vector<int32_t> prow(pl.sprow), pinv((size_t)pl.n, -1);
    for (int32_t c = 0; c < pl.n; c++) if (prow[(size_t)c] >= 0) pinv[(size_t)prow[(size_t)c]] = c;
    CU(cudaMemcpy(h->d.prow, prow.data(), (size_t)pl.n * 4, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->d.pinv, pinv.data(), (size_t)pl.n * 4, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->d.order, pl.sorder.data(), (size_t)pl.n * 4, cudaMemcpyHostToDevice));
    if (!h->d.iorder) TRY(upload(h, (int32_t **)&h->d.iorder, pl.iorder));
    CU(cudaMemcpy(h->d.level, pl.slevel.data(), (size_t)pl.n * 4, cudaMemcpyHostToDevice));
    return BASKER_OK;
}

// A device copy of the arena right after the symbolic pass: L/U patterns at
// their regions, region bounds, counts, natural pivots, the symbolic static
// schedule, an identity (the natural preferred rows) and the pool cursors.
int save_symbolic_image(basker_t h)
{
    const bk_plan &pl = h->pl;
    const size_t n = (size_t)pl.n;
    if (!h->sym_Li) {
        TRY(dalloc(h, &h->sym_Li, (size_t)std::max<int64_t>(pl.lcap, 1)));
        TRY(dalloc(h, &h->sym_Ui, (size_t)std::max<int64_t>(pl.ucap, 1)));
        TRY(dalloc(h, &h->sym_n, 8 * std::max<size_t>(n, 1)));
        TRY(dalloc(h, &h->sym_beg, 4 * std::max<size_t>(n, 1)));
        TRY(dalloc(h, &h->sym_pool, 2));
    }
    bk_dev &d = h->d;
    CU(cudaMemcpy(h->sym_Li, d.Li, sizeof(int32_t) * (size_t)pl.lcap, cudaMemcpyDeviceToDevice));
    CU(cudaMemcpy(h->sym_Ui, d.Ui, sizeof(int32_t) * (size_t)pl.ucap, cudaMemcpyDeviceToDevice));
    int32_t *const a[6] = {d.Lcnt, d.Ucnt, d.prow, d.pinv, d.order, d.level};
    for (int i = 0; i < 6; i++) CU(cudaMemcpy(h->sym_n + i * n, a[i], n * 4, cudaMemcpyDeviceToDevice));
    std::vector<int32_t> ident(n);
    for (size_t c = 0; c < n; c++) ident[c] = (int32_t)c;
    CU(cudaMemcpy(h->sym_n + 6 * n, ident.data(), n * 4, cudaMemcpyHostToDevice));
    int64_t *const b[4] = {d.Lbeg, d.Ubeg, d.Lend, d.Uend};
    for (int i = 0; i < 4; i++) CU(cudaMemcpy(h->sym_beg + i * n, b[i], n * 8, cudaMemcpyDeviceToDevice));
    CU(cudaMemcpy(h->sym_pool, d.pool, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice));
    h->sym_ver = h->arena_ver;
    return BASKER_OK;
}

int restore_symbolic_image(basker_t h, cudaStream_t s)
{
    const bk_plan &pl = h->pl;
    const size_t n = (size_t)pl.n;
    bk_dev &d = h->d;
    CU(cudaMemcpyAsync(d.Li, h->sym_Li, sizeof(int32_t) * (size_t)pl.lcap, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(d.Ui, h->sym_Ui, sizeof(int32_t) * (size_t)pl.ucap, cudaMemcpyDeviceToDevice, s));
    int32_t *const a[7] = {d.Lcnt, d.Ucnt, d.prow, d.pinv, d.order, d.level, const_cast<int32_t *>(d.pref)};
    for (int i = 0; i < 7; i++) CU(cudaMemcpyAsync(a[i], h->sym_n + i * n, n * 4, cudaMemcpyDeviceToDevice, s));
    int64_t *const b[4] = {d.Lbeg, d.Ubeg, d.Lend, d.Uend};
    for (int i = 0; i < 4; i++) CU(cudaMemcpyAsync(b[i], h->sym_beg + i * n, n * 8, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(d.pool, h->sym_pool, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
    return BASKER_OK;
}

int setup_device(basker_t h)
{
    bk_plan &pl = h->pl;
    bk_dev &d = h->d;
    const int32_t n = pl.n;
    d.n = n;
    d.ntasks = (int32_t)pl.tasks.size();
    d.prec = h->opt.precision == 1 ? 1 : 0;     // precision 2: FP64 factors, refined solves
    if (h->opt.precision >= 1) {
        // B by rows (entries in ascending column order) for the FP64 residual
        std::vector<int64_t> brp((size_t)n + 1, 0);
        for (int32_t j = 0; j < n; j++)
            for (int32_t e = pl.Bp[(size_t)j]; e < pl.Bp[(size_t)j + 1]; e++) brp[(size_t)pl.Bi[(size_t)e] + 1]++;
        for (int32_t i = 0; i < n; i++) brp[(size_t)i + 1] += brp[(size_t)i];
        std::vector<int32_t> brj((size_t)pl.nnz), brpos((size_t)pl.nnz), blk((size_t)n, 0);
        std::vector<int64_t> cur(brp.begin(), brp.end() - 1);
        for (int32_t j = 0; j < n; j++)
            for (int32_t e = pl.Bp[(size_t)j]; e < pl.Bp[(size_t)j + 1]; e++) {
                const int64_t q = cur[(size_t)pl.Bi[(size_t)e]]++;
                brj[(size_t)q] = j;
                brpos[(size_t)q] = e;
            }
        for (int32_t b = 0; b < pl.nblocks; b++)
            for (int32_t i = pl.block_ptr[(size_t)b]; i < pl.block_ptr[(size_t)b + 1]; i++) blk[(size_t)i] = b;
        TRY(upload(h, (int64_t **)&h->rf.Brp, brp));
        TRY(upload(h, (int32_t **)&h->rf.Brj, brj));
        TRY(upload(h, (int32_t **)&h->rf.Brpos, brpos));
        TRY(upload(h, (int32_t **)&h->rf.blk, blk));
        TRY(dalloc(h, &h->rf.Bx64, (size_t)pl.nnz));
        TRY(dalloc(h, &h->rf.bmax, (size_t)std::max(pl.nblocks, 1)));
        TRY(dalloc(h, &h->rf.umax, (size_t)std::max(pl.nblocks, 1)));
        TRY(dalloc(h, &h->d_norms, 2));
        TRY(dalloc(h, &h->d_vals64, (size_t)pl.nnz));
        CU(cudaMallocHost((void **)&h->h_norms, sizeof(double) * 2));
    }
    TRY(upload(h, (int32_t **)&d.Bp, pl.Bp));
    TRY(upload(h, (int32_t **)&d.Bi, pl.Bi));
    TRY(upload(h, (int32_t **)&d.dstart, pl.dstart));
    TRY(upload(h, (int32_t **)&d.bmap, pl.bmap));
    TRY(upload(h, (int32_t **)&d.col_task, pl.col_task));
    TRY(dalloc(h, &d.Bx, (size_t)pl.nnz, true));
    // every separator fits the dense elimination: refactorizations recompute the
    // separators by it, after the stored-pattern pass and rounds of the ND leaves
    // and BTF blocks (a separator's in-node chain is the long part of the
    // stored-pattern pass, and any change below a separator redoes it anyway)
    h->sep_dense = false;
    if (h->opt.factor_mode == 0) {
        bool all = true, any = false;
        for (const bk_task &T : pl.tasks)
            if (T.sp_lo < T.lo) {
                any = true;
                all = all && bk_dense_node_eligible(T);
            }
        h->sep_dense = any && all;
    }
    for (bk_task &T : pl.tasks) T.dense = (h->sep_dense && T.sp_lo < T.lo) ? 1 : 0;
    TRY(upload(h, &d.tasks, pl.tasks));
    if (h->sep_dense) {
        std::vector<int32_t> ids;
        for (size_t t = 0; t < pl.tasks.size(); t++)
            if (!pl.tasks[t].dense) ids.push_back((int32_t)t);
        TRY(upload(h, &h->rp_tasks, ids));
        h->rp_ntasks = (int32_t)ids.size();
        h->rp_smem = bk_repair_smem(pl.tasks.data(), ids.data(), (int32_t)ids.size(), 160 * 1024);
        h->rp_ctas = std::max(1, std::min<int>({h->rp_ntasks, pl.wsd_warps, 152 * 8}));
    }
    TRY(dalloc(h, &d.prow, (size_t)n));
    TRY(dalloc(h, &d.pinv, (size_t)n));
    TRY(dalloc(h, (int32_t **)&d.pref, (size_t)n));
    TRY(dalloc(h, &d.Lcnt, (size_t)n, true));
    TRY(dalloc(h, &d.Ucnt, (size_t)n, true));
    TRY(dalloc(h, &d.pool, 2, true));
    TRY(alloc_factors(h));
    TRY(dalloc(h, &d.status, 1, true));
    TRY(dalloc(h, &d.col_over, (size_t)n, true));
    TRY(dalloc(h, &d.task_stop, pl.tasks.size(), true));
    TRY(dalloc(h, &d.task_fail, pl.tasks.size()));
    TRY(dalloc(h, &d.col_fail, (size_t)n, true));
    TRY(dalloc(h, &d.dd_start, pl.tasks.size(), true));
    TRY(dalloc(h, &d.dd_flags, pl.tasks.size(), true));
    TRY(dalloc(h, &d.touch, (size_t)n, true));
    TRY(dalloc(h, &d.dirty_ep, (size_t)n, true));
    TRY(dalloc(h, &d.pchg_ep, (size_t)n, true));
    TRY(dalloc(h, &d.touch_ref, (size_t)n, true));
    TRY(dalloc(h, &d.dirty_ref, (size_t)n, true));
    TRY(dalloc(h, &d.pchg_ref, (size_t)n, true));
    TRY(dalloc(h, &d.ws, (size_t)std::max<int64_t>(pl.ws_bytes, 256), true));
    TRY(dalloc(h, &d.done, (size_t)n, true));
    TRY(dalloc(h, &d.order, (size_t)n));
    TRY(dalloc(h, &d.counter, 8, true));
    TRY(dalloc(h, &d.level, (size_t)n * 2 + 2, true));
    TRY(dalloc(h, &d.ahat, (size_t)pl.ahat_doubles));
    TRY(dalloc(h, &d.abits, (size_t)pl.ahat_words));
    TRY(dalloc(h, &d.dcnt, (size_t)n, true));
    d.wsd_slice = pl.wsd_slice;
    d.wsd_warps = pl.wsd_warps;
    d.dd_words = pl.dd_words;
    TRY(dalloc(h, &d.wsd, (size_t)pl.wsd_bytes, true));
    d.sx_warps = bk_static_blocks() * 4;
    // x over the space of the tasks the stored-pattern pass computes (it leaves the
    // separators that the dense elimination recomputes)
    int32_t sx_space = 1;
    for (const bk_task &T : pl.tasks)
        if (!T.dense) sx_space = std::max(sx_space, T.space);
    d.sx_stride = ((int64_t)sx_space + 31) & ~(int64_t)31;
    TRY(dalloc(h, &d.sx, (size_t)(d.sx_stride * d.sx_warps), true));
    d.nblocks = pl.nblocks;
    TRY(upload(h, (int32_t **)&d.block_ptr, pl.block_ptr));
    TRY(upload(h, (int32_t **)&d.P, pl.P));
    TRY(upload(h, (int32_t **)&d.Q, pl.Q));
    // level lists of a full factorization
    const size_t nl = pl.level_tasks.size();
    h->lv_tasks.assign(nl, nullptr);
    h->lv_ntasks.assign(nl, 0);
    h->lv_smem.assign(nl, 0);
    h->lv_cols.assign(nl, nullptr);
    h->lv_ncols.assign(nl, 0);
    for (int g = 0; g < 2; g++) {
        h->lv_dense[g].assign(nl, nullptr);
        h->lv_ndense[g].assign(nl, 0);
        h->lv_dsmem[g].assign(nl, 0);
    }
    for (size_t l = 0; l < nl; l++) {
        std::vector<int32_t> ids, dense[2];
        size_t sm = 0, dsm[2] = {0, 0};
        std::vector<int32_t> cols;
        for (int32_t t : pl.level_tasks[l]) {
            const bk_task &T = pl.tasks[(size_t)t];
            if (h->opt.factor_mode == 0 && bk_dense_node_eligible(T)) {
                const int g = bk_dense_node_cluster(T) > 1 ? 1 : 0;
                dense[g].push_back(t);
                dsm[g] = std::max(dsm[g], bk_dense_node_smem(T));
            } else {
                ids.push_back(t);
                if (T.wsoff < 0) sm = std::max(sm, bk_task_smem_bytes(T));
            }
            if (T.sp_lo < T.lo)
                for (int32_t c = T.lo; c < T.hi; c++) cols.push_back(c);
        }
        TRY(upload(h, &h->lv_tasks[l], ids));
        h->lv_ntasks[l] = (int32_t)ids.size();
        for (int g = 0; g < 2; g++) {
            TRY(upload(h, &h->lv_dense[g][l], dense[g]));
            h->lv_ndense[g][l] = (int32_t)dense[g].size();
            h->lv_dsmem[g][l] = (dsm[g] + 15) & ~(size_t)15;
        }
        h->lv_smem[l] = (sm + 15) & ~(size_t)15;
        TRY(upload(h, &h->lv_cols[l], cols));
        h->lv_ncols[l] = (int32_t)cols.size();
    }
    TRY(dalloc(h, &h->rd_tasks, (size_t)std::max<size_t>(pl.tasks.size(), 1)));
    TRY(dalloc(h, &h->rd_c0, (size_t)std::max<size_t>(pl.tasks.size(), 1)));
    TRY(dalloc(h, &h->rd_cols, (size_t)std::max(n, 1)));
    TRY(dalloc(h, &h->df_redo, (size_t)std::max(n, 1)));
    h->df_par.clear();
    for (size_t l = 0; l < pl.level_tasks.size(); l++) h->df_par.push_back(bk_desc_fast_params(pl, (int32_t)l));
    CU(cudaMallocHost((void **)&h->h_stage, sizeof(int32_t) * ((size_t)n + 4 * pl.tasks.size() + 16)));
    CU(cudaMallocHost((void **)&h->h_status, sizeof(bk_status)));
    CU(cudaMallocHost((void **)&h->h_task_fail, sizeof(int32_t) * std::max<size_t>(pl.tasks.size(), 1)));
    // solve
    bk_solve_plan_build(pl, h->sp);
    bk_solve_dev &s = h->sd;
    s.nitems = (int32_t)h->sp.items.size();
    TRY(upload(h, &s.items, h->sp.items));
    s.nsweeps = (int32_t)h->sp.sweeps.size();
    TRY(upload(h, (int32_t **)&s.sweeps, h->sp.sweeps));
    bk_solve_sweep_setup(s, h->sp.sw_maxm);
    TRY(upload(h, (int32_t **)&s.offp, h->sp.offp));
    TRY(upload(h, (int32_t **)&s.offj, h->sp.offj));
    TRY(upload(h, (int32_t **)&s.offpos, h->sp.offpos));
    TRY(upload(h, (int32_t **)&s.cutlo, h->sp.cutlo));
    TRY(upload(h, (int32_t **)&s.cuthi, h->sp.cuthi));
    s.nleaves = (int32_t)h->sp.leaf_tasks.size();
    s.leaf_rows = h->sp.leaf_rows;
    s.leaf_f0 = h->sp.leaf_f0;
    s.leaf_b0 = h->sp.leaf_b0;
    s.leaf_maxrows = h->sp.leaf_maxrows;
    TRY(upload(h, (int32_t **)&s.leaf_tasks, h->sp.leaf_tasks));
    TRY(dalloc(h, &s.leaf_bad, std::max<size_t>(h->sp.leaf_tasks.size(), 1)));
    TRY(dalloc(h, &s.lcnt, (size_t)2 * ((size_t)h->sp.leaf_maxrows + 1)));
    TRY(dalloc(h, &s.fdone, (size_t)n, true));
    TRY(dalloc(h, &s.bdone, (size_t)n, true));
    TRY(dalloc(h, &s.r.Lrp, (size_t)n + 1));
    TRY(dalloc(h, &s.r.Urp, (size_t)n + 1));
    TRY(dalloc(h, &s.r.Ud, (size_t)n));
    TRY(dalloc(h, &s.r.cnt, (size_t)2 * ((size_t)n + 1)));
    TRY(dalloc(h, &s.r.part, (size_t)n / 1024 + 2));
    s.r.swords = (int64_t)n / 32 + 2;
    TRY(dalloc(h, &s.r.longs, (size_t)n + 1));
    TRY(dalloc(h, &s.r.sbits, (size_t)(s.r.swords * BK_LONG_CTAS)));
    TRY(dalloc(h, &s.r.spre, (size_t)(s.r.swords * BK_LONG_CTAS)));
    TRY(upload_symbolic_pattern(h));
    if (!pl.counts_only) TRY(save_symbolic_image(h));
    h->schedule_valid = !pl.counts_only;
#ifdef BK_TRACE
    TRY(dalloc(h, &d.trace, (size_t)4 + 4 * (size_t)BK_TRACE_CAP, true));
#endif
    return BASKER_OK;
}

// launch_redo's answer when the rest of a refactorization is cheaper as one complete pass
constexpr int BK_SWITCH_TO_FULL = -2;
// rounds of at least this many columns give the cost per column the switch predicts with
constexpr size_t BK_ROUND_LARGE = 100000;

int reset_status(basker_t h, cudaStream_t s)
{
    CU(cudaMemsetAsync(h->d.status, 0, sizeof(bk_status), s));
    CU(cudaMemsetAsync(h->d.task_stop, 0, sizeof(int32_t) * std::max<size_t>(h->pl.tasks.size(), 1), s));
    CU(cudaMemsetAsync(&h->d.status->first_fail, 0xff, sizeof(unsigned long long), s));
    if (h->ws_dirty) {
        CU(cudaMemsetAsync(h->d.ws, 0, (size_t)std::max<int64_t>(h->pl.ws_bytes, 256), s));
        CU(cudaMemsetAsync(h->d.wsd, 0, (size_t)h->pl.wsd_bytes, s));
        CU(cudaMemsetAsync(h->d.sx, 0, sizeof(double) * (size_t)(h->d.sx_stride * h->d.sx_warps), s));
        h->ws_dirty = false;
    }
    return BASKER_OK;
}

// Read the status word; translate failures.  Returns OK, SINGULAR, NAN, TIMEOUT,
// or -1 for a capacity overflow (the caller regrows).
int read_status(basker_t h, cudaStream_t s)
{
    CU(cudaMemcpyAsync(h->h_status, h->d.status, sizeof(bk_status), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    CU(cudaGetLastError());
    const bk_status &st = *h->h_status;
    h->info.failed_column = -1;
    if (st.timeout) { h->ws_dirty = true; return BASKER_ERR_TIMEOUT; }
    // an overflow stops its task midway, which later kernels may see as an
    // inconsistency: the regrow and full recomputation come first
    if (st.capacity) { h->ws_dirty = true; return -1; }
    if (st.first_fail != ~0ull) {
        h->ws_dirty = true;
        h->info.failed_column = (int32_t)(st.first_fail >> 8);
        const unsigned code = (unsigned)(st.first_fail & 0xff);
        if (code == BK_CODE_INTERNAL) {
            h->info.internal_site = st.internal_site;
            h->info.internal_col = st.internal_col;
            return BASKER_ERR_INVALID_ARG;
        }
        return code == BK_CODE_NAN ? BASKER_ERR_NAN : BASKER_ERR_SINGULAR;
    }
    if (st.capacity) { h->ws_dirty = true; return -1; }
    return BASKER_OK;
}

int regrow(basker_t h)
{
    std::vector<int32_t> over((size_t)h->pl.n);
    CU(device_sync());
    CU(cudaMemcpy(over.data(), h->d.col_over, over.size() * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemset(h->d.col_over, 0, over.size() * 4));
    bk_plan_regrow(h->pl, over.data());
    TRY(alloc_factors(h));
    h->info.capacity_regrows++;
    h->ws_dirty = true;
    return BASKER_OK;
}

// The handle's device view with the column-per-warp workspace cut into the
// slices of ND level l (one workspace serves the levels in turn).
bk_dev level_dev(basker_t h, size_t l)
{
    bk_dev d = h->d;
    if (l < h->pl.level_slice.size()) {
        d.wsd_slice = h->pl.level_slice[l];
        d.wsd_warps = h->pl.level_warps[l];
    }
    if (l < h->pl.level_dd_words.size()) d.dd_words = h->pl.level_dd_words[l];
    return d;
}

// The descendant phase of separator columns cols[0..ncols) of ND level `level` in
// a refactorization: first on their stored patterns (verified on the device),
// then the reach kernel over the columns that failed (their list and count stay
// on the device).
int launch_desc_refactor(basker_t h, const int32_t *cols, int32_t ncols, cudaStream_t s, size_t level)
{
    if (ncols <= 0) return BASKER_OK;
    const bk_dev dl = level_dev(h, level);
    CU(cudaMemsetAsync(h->d.counter + 5, 0, sizeof(int32_t), s));
    CU(cudaMemsetAsync(h->d.counter + 7, 0, sizeof(int32_t), s));
    CU(cudaMemsetAsync(h->d.counter + 3, 0, sizeof(int32_t), s));
    const bk_desc_par par = level < h->df_par.size() ? h->df_par[level] : bk_desc_par{};
    if (!par.smem) {
        // separators too large for the stored-pattern kernel: every column by the reach
        tbeg(h, KT_DESC, s, 1);
        bk_launch_gp_desc(dl, cols, ncols, h->d.counter + 3, s);
        CU(cudaGetLastError());
        tend(h, s);
        h->launches++;
        return BASKER_OK;
    }
    tbeg(h, KT_DESC, s, 2);
    bk_launch_desc_fast(dl, cols, ncols, h->d.counter + 5, h->df_redo, h->d.counter + 7, par, s);
    CU(cudaGetLastError());
    bk_launch_gp_desc(dl, h->df_redo, ncols, h->d.counter + 3, s, h->d.counter + 7);
    CU(cudaGetLastError());
    tend(h, s);
    h->launches += 2;
    return BASKER_OK;
}

// Algorithm 1 on every task, level by level (Algorithm 4's dependency tree).
int launch_full_gp(basker_t h, cudaStream_t s, int pref_mode)
{
    const double tau = h->opt.tau;
    CU(cudaMemsetAsync(h->d.pinv, 0xff, sizeof(int32_t) * (size_t)h->pl.n, s));
    for (size_t l = 0; l < h->lv_tasks.size(); l++) {
        if (l > 0 && h->lv_ncols[l] > 0) {
            CU(cudaMemsetAsync(h->d.counter + 3, 0, sizeof(int32_t), s));
            tbeg(h, KT_DESC, s, 1);
            bk_launch_gp_desc(level_dev(h, l), h->lv_cols[l], h->lv_ncols[l], h->d.counter + 3, s);
            CU(cudaGetLastError());
            tend(h, s);
            h->launches++;
        }
        if (h->lv_ntasks[l] > 0) {
            tbeg(h, KT_GP, s, 1);
            bk_launch_gp_tasks(h->d, h->lv_tasks[l], nullptr, h->lv_ntasks[l], h->lv_smem[l], tau, pref_mode, s);
            CU(cudaGetLastError());
            tend(h, s);
            h->launches++;
        }
        for (int g = 0; g < 2; g++) {
            if (h->lv_ndense[g][l] == 0) continue;
            tbeg(h, KT_DENSE, s, 1);
            bk_launch_dense_nodes(h->d, h->lv_dense[g][l], h->lv_ndense[g][l], h->lv_dsmem[g][l], tau, pref_mode,
                                  g ? BK_DENSE_CLUSTER : 1, s);
            CU(cudaGetLastError());
            tend(h, s);
            h->launches++;
        }
    }
    CU(cudaGetLastError());
    return BASKER_OK;
}

// Upload a list of ints through the pinned staging buffer (at offset off ints).
int stage_upload(basker_t h, cudaStream_t s, int32_t *dst, const std::vector<int32_t> &v, size_t off)
{
    if (v.empty()) return BASKER_OK;
    std::memcpy(h->h_stage + off, v.data(), v.size() * 4);
    CU(cudaMemcpyAsync(dst, h->h_stage + off, v.size() * 4, cudaMemcpyHostToDevice, s));
    return BASKER_OK;
}

// The columns of a round in claim order (bk_round_order): each active task's
// columns from its start column on.
void round_columns(const bk_plan &pl, const std::vector<int32_t> &active, const std::vector<int32_t> &start,
                   std::vector<int32_t> &cols)
{
    std::vector<std::pair<int32_t, int32_t>> ranges;
    ranges.reserve(active.size());
    for (int32_t t : active) ranges.emplace_back(start[(size_t)t], pl.tasks[(size_t)t].hi);
    bk::bk_round_order(ranges, cols);
}

// After a stored-pattern pass that rejected some preferred pivots (first
// rejection per task in h_task_fail): level by level up the ND tree, rounds of the
// dirty-dataflow kernel.  A task with a rejected column f starts a round at f
// (resolve); a separator whose descendants changed starts at its first column
// (force); after a round, each task that rejected a speculated pivot at f' runs
// another round from f'.  Separators whose in-node phase fits the dense
// elimination are instead recomputed whole: descendant phase, then the dense
// elimination with the previous pivots preferred (the refactorization's
// definition for those columns, as in a complete pass).
int launch_redo(basker_t h, cudaStream_t s)
{
    bk_plan &pl = h->pl;
    const double tau = h->opt.tau;
    const size_t nt = pl.tasks.size();
    std::vector<int32_t> fail(h->h_task_fail, h->h_task_fail + nt);
    std::vector<char> desc_changed(nt, 0);
    std::vector<int32_t> start(nt, 0), flags(nt, 0);
    int32_t redone = 0;
    h->info.last_rounds = 0;
    const auto t0 = std::chrono::steady_clock::now();
    auto mark_ancestors = [&](size_t t) {
        const bk_task &T = pl.tasks[t];
        for (int32_t a = 0; a < T.nanc; a++) desc_changed[(size_t)pl.col_task[(size_t)T.anc_lo[a]]] = 1;
    };
    for (size_t l = 0; l < pl.level_tasks.size(); l++) {
        std::vector<int32_t> active;
        for (int32_t t : pl.level_tasks[l]) {
            const bk_task &T = pl.tasks[(size_t)t];
            if (T.dense) {
                active.push_back(t);
                start[(size_t)t] = T.lo;
                flags[(size_t)t] = BK_DD_DESC;
            } else if (desc_changed[(size_t)t]) {
                active.push_back(t);
                start[(size_t)t] = T.lo;
                flags[(size_t)t] = BK_DD_DESC;
            } else if (fail[(size_t)t] >= T.lo && fail[(size_t)t] < T.hi) {
                active.push_back(t);
                start[(size_t)t] = fail[(size_t)t];
                flags[(size_t)t] = BK_DD_RESOLVE;
            }
        }
        for (int32_t t : active) mark_ancestors((size_t)t);
        if (l > 0 && h->sep_dense && !active.empty()) {
            // separators: the descendant phase and one dense elimination with the
            // previous pivots preferred recompute each of them in two launches,
            // instead of rounds of column-by-column recomputation.  All or none:
            // the rounds of a separator rely on the change markers that rounds
            // leave on the columns below it, which the dense path does not set.
            std::vector<int32_t> dense[2], rest, cols;
            size_t dsm[2] = {0, 0};
            for (int32_t t : active) {
                const bk_task &T = pl.tasks[(size_t)t];
                if (bk_dense_node_eligible(T)) {
                    const int g = bk_dense_node_cluster(T) > 1 ? 1 : 0;
                    dense[g].push_back(t);
                    dsm[g] = std::max(dsm[g], bk_dense_node_smem(T));
                    for (int32_t c = T.lo; c < T.hi; c++) cols.push_back(c);
                } else {
                    rest.push_back(t);
                }
            }
            if (!cols.empty()) {
                CU(cudaStreamSynchronize(s));       // the staging buffer is reused
                TRY(stage_upload(h, s, h->rd_cols, cols, 0));
                TRY(stage_upload(h, s, h->rd_tasks, dense[0], (size_t)pl.n));
                TRY(stage_upload(h, s, h->rd_tasks + dense[0].size(), dense[1], (size_t)pl.n + dense[0].size()));
                TRY(launch_desc_refactor(h, h->rd_cols, (int32_t)cols.size(), s, l));
                for (int g = 0; g < 2; g++) {
                    if (dense[g].empty()) continue;
                    tbeg(h, KT_DENSE, s, 1);
                    bk_launch_dense_nodes(h->d, h->rd_tasks + (g ? dense[0].size() : 0), (int32_t)dense[g].size(),
                                          (dsm[g] + 15) & ~(size_t)15, tau, 1, g ? BK_DENSE_CLUSTER : 1, s);
                    CU(cudaGetLastError());
                    tend(h, s);
                    h->launches++;
                }
                h->launches++;
                h->info.last_rounds++;
                redone += (int32_t)cols.size();
                const int st = read_status(h, s);
                if (st != BASKER_OK) return st;
            }
            active.swap(rest);
        }
        for (int round = 0; !active.empty(); round++) {
            if (round > 4 * (int)pl.n + 8) return BASKER_ERR_INVALID_ARG;   // cannot happen: each round resolves a column
            std::vector<int32_t> cols;
            round_columns(pl, active, start, cols);
            // a large round that would, at the cost per column of the large rounds
            // seen so far, take the rounds past a complete pass: the complete pass now
            // instead (small rounds are dominated by their fixed costs: not predicted)
            const double limit0 = h->gp_wall_ms > 0.0 ? h->gp_wall_ms : 20.0 * h->static_factor_ms;
            const double spent = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if ((h->opt.refactor_switch == 0 || h->opt.refactor_switch == 3) && limit0 > 0.0 &&
                h->round_us_per_col > 0.0 && cols.size() >= BK_ROUND_LARGE &&
                spent + 1e-3 * h->round_us_per_col * (double)cols.size() > limit0) {
                h->info.last_repivot_columns = redone;
                return BK_SWITCH_TO_FULL;
            }
            const auto tr = std::chrono::steady_clock::now();
            CU(cudaStreamSynchronize(s));       // the staging buffer is reused
            std::memcpy(h->h_stage, start.data(), nt * 4);
            std::memcpy(h->h_stage + nt, flags.data(), nt * 4);
            CU(cudaMemcpyAsync(h->d.dd_start, h->h_stage, nt * 4, cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(h->d.dd_flags, h->h_stage + nt, nt * 4, cudaMemcpyHostToDevice, s));
            TRY(stage_upload(h, s, h->rd_cols, cols, 2 * nt));
            CU(cudaMemsetAsync(h->d.task_fail, 0x7f, sizeof(int32_t) * nt, s));
            CU(cudaMemsetAsync(h->d.counter + 3, 0, sizeof(int32_t), s));
            h->epoch++;
            tbeg(h, KT_SPEC, s, 1);
            bk_launch_dd(level_dev(h, l), h->rd_cols, (int32_t)cols.size(), h->d.counter + 3, tau, h->epoch,
                         h->opt.wait_budget_cycles, h->refno, s, h->tune_dd);
            CU(cudaGetLastError());
            tend(h, s);
            h->launches++;
            h->info.last_rounds++;
            redone += (int32_t)cols.size();
            h->info.rounds_columns += (int64_t)cols.size();
            CU(cudaMemcpyAsync(h->h_task_fail, h->d.task_fail, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, s));
            const int st = read_status(h, s);
            if (st != BASKER_OK) return st;
            if (cols.size() >= BK_ROUND_LARGE) {
                const double us = 1e3 * std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tr).count() /
                                  (double)cols.size();
                h->round_us_per_col = h->round_us_per_col > 0.0 ? 0.5 * (h->round_us_per_col + us) : us;
            }
            std::vector<int32_t> next;
            for (int32_t t : active) {
                const bk_task &T = pl.tasks[(size_t)t];
                const int32_t f = h->h_task_fail[(size_t)t];
                if (f >= T.lo && f < T.hi) {
                    next.push_back(t);
                    start[(size_t)t] = f;
                    flags[(size_t)t] = BK_DD_RESOLVE;
                }
            }
            active.swap(next);
            // the rounds have cost as much as a complete pass would: finish with one
            // (no complete pass timed yet: twenty stored-pattern factorizations)
            const double limit = h->gp_wall_ms > 0.0 ? h->gp_wall_ms : 20.0 * h->static_factor_ms;
            if (!active.empty() && (h->opt.refactor_switch == 0 || h->opt.refactor_switch == 3) && limit > 0.0 &&
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > limit) {
                h->info.last_repivot_columns = redone;
                return BK_SWITCH_TO_FULL;
            }
        }
    }
    h->info.last_repivot_columns = redone;
    CU(cudaGetLastError());
    return BASKER_OK;
}

// The repair pass serves refactorizations with options.refactor_switch 3 whose
// separators are all recomputed densely.
bool use_repair(basker_t h) { return h->sep_dense && h->opt.refactor_switch == 3 && h->rp_ntasks > 0; }

// Counters of the last repair pass (from the status word just read).
void note_repair(basker_t h)
{
    const int32_t rep = h->h_status->repaired;
    h->info.last_repivot_columns = rep;
    h->info.last_rounds = rep > 0 ? 1 : 0;
    h->info.rounds_columns += rep;
}

// After a stored-pattern pass, when every separator is recomputed densely: the
// repair pass over the ND leaves and BTF blocks (each task with a rejected pivot
// walks its columns from the first rejection on, on the device), then each ND
// level's separators by the descendant phase and the dense elimination with the
// previous pivots preferred.  Asynchronous: nothing is read back here.
int launch_repair_path(basker_t h, cudaStream_t s)
{
    CU(cudaMemsetAsync(h->d.counter + 4, 0, sizeof(int32_t), s));
    tbeg(h, KT_SPEC, s, 1);
    bk_launch_repair(h->d, h->rp_tasks, h->rp_ntasks, h->d.counter + 4, h->opt.tau, h->rp_smem, h->rp_ctas, s);
    CU(cudaGetLastError());
    tend(h, s);
    h->launches++;
    for (size_t l = 1; l < h->lv_tasks.size(); l++) {
        TRY(launch_desc_refactor(h, h->lv_cols[l], h->lv_ncols[l], s, l));
        for (int g = 0; g < 2; g++) {
            if (h->lv_ndense[g][l] == 0) continue;
            tbeg(h, KT_DENSE, s, 1);
            bk_launch_dense_nodes(h->d, h->lv_dense[g][l], h->lv_ndense[g][l], h->lv_dsmem[g][l], h->opt.tau, 1,
                                  g ? BK_DENSE_CLUSTER : 1, s);
            CU(cudaGetLastError());
            tend(h, s);
            h->launches++;
        }
    }
    return BASKER_OK;
}

int compute_schedule(basker_t h, cudaStream_t s)
{
    h->epoch++;
    tbeg(h, KT_LEVELS, s, 5);
    // the stored levels are kept when they still order the new pattern (checked on
    // the device: a refactorization usually changes few columns)
    bk_launch_levels(h->d, h->epoch, h->opt.wait_budget_cycles, static_blocks(h), s, true);
    CU(cudaGetLastError());
    tend(h, s);
    h->launches += 5;
    CU(cudaGetLastError());
    h->schedule_valid = true;
    h->order_is_symbolic = false;
    return BASKER_OK;
}

int static_pass(basker_t h, cudaStream_t s)
{
    CU(cudaMemsetAsync(h->d.task_fail, 0x7f, sizeof(int32_t) * h->pl.tasks.size(), s));
    CU(cudaMemsetAsync(h->d.counter, 0, sizeof(int32_t), s));
    h->epoch++;
    tbeg(h, KT_STATIC, s, 1);
    bk_launch_static(h->d, h->pl.n, h->opt.tau, h->epoch, h->opt.wait_budget_cycles, static_blocks(h), s);
    CU(cudaGetLastError());
    tend(h, s);
    h->launches++;
    CU(cudaGetLastError());
    return BASKER_OK;
}

// After a factorization: the column levels of the new pattern (the next
// refactorization's claim order, and the backward order of the ND leaves in the
// solve), the factors by rows, and the solve's order of the leaf rows.
// The factors into rows and the solve's leaf order: 19 launches that depend on
// nothing but the arena, recorded once into a CUDA graph (on the handle's own
// stream, so that the caller's stream may be the legacy default stream) and
// replayed on the caller's stream.
int capture_finish(basker_t h)
{
    if (!h->cap_stream) CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (h->g_finish) {
        cudaGraphExecDestroy(h->g_finish);
        h->g_finish = nullptr;
    }
    cudaGraph_t g = nullptr;
    std::lock_guard<std::mutex> lk(g_capture_mu);
    CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    bk_launch_rows(h->d, h->sd.r, h->cap_stream);
    bk_launch_leaf_order(h->d, h->sd, h->cap_stream);
    CU(cudaStreamEndCapture(h->cap_stream, &g));
    const cudaError_t e = cudaGraphInstantiate(&h->g_finish, g, 0);
    cudaGraphDestroy(g);
    CU(e);
    h->g_finish_ver = h->arena_ver;
    return BASKER_OK;
}

int finish_factorization(basker_t h, cudaStream_t s)
{
    if (!h->schedule_valid) TRY(compute_schedule(h, s));
    tbeg(h, KT_ROWS, s, 19);
    if (h->opt.graphs) {
        if (!h->g_finish || h->g_finish_ver != h->arena_ver) TRY(capture_finish(h));
        CU(cudaGraphLaunch(h->g_finish, s));
        h->info.graph_launches++;
    } else {
        bk_launch_rows(h->d, h->sd.r, s);
        CU(cudaGetLastError());
        bk_launch_leaf_order(h->d, h->sd, s);
    }
    CU(cudaGetLastError());
    tend(h, s);
    CU(cudaGetLastError());
    return BASKER_OK;
}

// A factorization by the refactorization's path: the symbolic arena (natural
// pivots preferred, the symbolic pattern and schedule) restored, the
// stored-pattern pass, rounds for the rejected natural pivots, the separators'
// dense recomputation.  This is Algorithm 1 with the natural rows preferred, the
// factorization's definition.  Returns BK_SWITCH_TO_FULL when the complete pass
// should run instead: no valid image, too many rejected pivots (the rounds would
// cost more than the pass; the handle then stops trying), or any other status (a failure, which the complete
// pass names exactly; a wait that gave up; an exhausted spill pool).
int factor_static(basker_t h, cudaStream_t s)
{
    if (!h->sym_Li || h->sym_ver != h->arena_ver || h->opt.factor_mode != 0 || h->static_factor_off)
        return BK_SWITCH_TO_FULL;
    const auto t0 = std::chrono::steady_clock::now();
    TRY(restore_symbolic_image(h, s));
    h->refno++;
    h->schedule_valid = true;
    h->order_is_symbolic = true;
    TRY(static_pass(h, s));
    CU(cudaMemcpyAsync(h->h_task_fail, h->d.task_fail, sizeof(int32_t) * h->pl.tasks.size(),
                       cudaMemcpyDeviceToHost, s));
    int st = read_status(h, s);
    if (st != BASKER_OK) return BK_SWITCH_TO_FULL;
    const int rejected = h->h_status->static_fail;
    if (rejected > std::max(16, h->pl.n / 200)) {
        h->static_factor_off = true;         // this pattern's values do not keep their natural pivots
        return BK_SWITCH_TO_FULL;
    }
    h->info.last_repivot_columns = 0;
    h->info.last_rounds = 0;
    if (rejected || h->sep_dense) {
        st = use_repair(h) ? launch_repair_path(h, s) : launch_redo(h, s);
        if (st == BASKER_OK) st = read_status(h, s);
        if (st != BASKER_OK) return BK_SWITCH_TO_FULL;
        if (use_repair(h)) note_repair(h);
        h->schedule_valid = false;
    }
    h->static_factor_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return BASKER_OK;
}

// A refactorization's rejected pivots by rounds of the round kernel (host-driven
// level by level; options.refactor_switch decides when the rest becomes one
// complete pass), after the stored-pattern pass.  Returns the final status
// (-1: the factors need more room even after the regrows).
int refactor_by_rounds(basker_t h, cudaStream_t s)
{
    CU(cudaMemcpyAsync(h->h_task_fail, h->d.task_fail, sizeof(int32_t) * h->pl.tasks.size(),
                       cudaMemcpyDeviceToHost, s));
    int st = read_status(h, s);
    if (st == BASKER_ERR_TIMEOUT) return st;
    if (!h->h_status->static_fail && !h->sep_dense) return st;
    // the complete pass at once (mode 2, or, by default, when the stored-pattern pass
    // rejected so many pivots that the rounds' cascades would recompute most columns
    // anyway: the same bound the factorization's path uses)
    const int rejected = h->h_status->static_fail;
    const bool full_now = rejected && (h->opt.refactor_switch == 2 ||
                                       (h->opt.refactor_switch == 0 && rejected > std::max(16, h->pl.n / 200)));
    st = full_now ? BK_SWITCH_TO_FULL : launch_redo(h, s);
    if (st == BASKER_OK) st = read_status(h, s);
    h->schedule_valid = false;
    if (st == BK_SWITCH_TO_FULL) {
        // Algorithm 1 on every column with the previous pivots preferred: the
        // refactorization's definition, computed directly
        h->info.full_refactors++;
        h->ws_dirty = true;
        TRY(reset_status(h, s));
        const auto t0 = std::chrono::steady_clock::now();
        TRY(launch_full_gp(h, s, 1));
        st = read_status(h, s);
        if (st == BASKER_OK)
            h->gp_wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    for (int tries = 0; st == -1 && tries < 16; tries++) {
        // the new pivots need more room: grow and run Algorithm 1 everywhere
        TRY(regrow(h));
        TRY(reset_status(h, s));
        TRY(launch_full_gp(h, s, 1));
        st = read_status(h, s);
    }
    return st;
}

int factor_impl(basker_t h, const double *values, cudaStream_t s, bool refactor)
{
    h->launches = 0;
    TRY(reset_status(h, s));
    tbeg(h, KT_GATHER, s, 1);
    bk_launch_gather(h->d, values, h->pl.nnz, s);
    CU(cudaGetLastError());
    tend(h, s);
    h->launches++;
    if (refactor) {
        h->refno++;
        CU(cudaMemcpyAsync((void *)h->d.pref, h->d.prow, sizeof(int32_t) * (size_t)h->pl.n,
                           cudaMemcpyDeviceToDevice, s));
        if (!h->schedule_valid) TRY(compute_schedule(h, s));
        TRY(static_pass(h, s));
        h->info.last_repivot_columns = 0;
        h->info.last_rounds = 0;
        int st = BASKER_OK;
        if (use_repair(h)) {
            // the stored-pattern pass, the repair pass and the separators run back to
            // back on the device; the status is read once at the end
            TRY(launch_repair_path(h, s));
            st = read_status(h, s);
            h->schedule_valid = false;
            if (st == BASKER_OK) note_repair(h);
            for (int tries = 0; st == -1 && tries < 16; tries++) {
                // the new pivots need more room: grow and run Algorithm 1 everywhere
                TRY(regrow(h));
                TRY(reset_status(h, s));
                TRY(launch_full_gp(h, s, 1));
                st = read_status(h, s);
            }
        } else {
            st = refactor_by_rounds(h, s);
            if (st == BASKER_ERR_TIMEOUT) return st;
        }
        if (st != BASKER_OK) { h->factored = false; return st == -1 ? BASKER_ERR_OOM : st; }
        TRY(finish_factorization(h, s));
        h->factored = true;
        return BASKER_OK;
    }
    int st = factor_static(h, s);
    if (st == BASKER_OK) {
        h->info.static_factors++;
        TRY(finish_factorization(h, s));
        h->factored = true;
        return BASKER_OK;
    }
    h->ws_dirty = true;
    TRY(reset_status(h, s));
    st = -1;
    for (int tries = 0; tries < 16; tries++) {
        if (tries > 0) {
            TRY(regrow(h));
            TRY(reset_status(h, s));
            tbeg(h, KT_GATHER, s, 1);
            bk_launch_gather(h->d, values, h->pl.nnz, s);
            CU(cudaGetLastError());
            tend(h, s);
        }
        const auto t0 = std::chrono::steady_clock::now();
        TRY(launch_full_gp(h, s, 0));
        st = read_status(h, s);
        if (st == BASKER_OK)
            h->gp_wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (st != -1) break;
    }
    if (st != BASKER_OK) { h->factored = false; return st == -1 ? BASKER_ERR_OOM : st; }
    // with the natural pivots everywhere the pattern is the symbolic one, whose
    // static schedule is already on the device
    h->schedule_valid = (h->h_status->offdiag == 0 && h->order_is_symbolic);
    TRY(finish_factorization(h, s));
    h->factored = true;
    return BASKER_OK;
}

int ensure_solve_buffers(basker_t h, int32_t nrhs)
{
    if (nrhs <= h->nrhs_cap) return BASKER_OK;
    dfree(h, h->sd.w);
    dfree(h, h->sd.z);
    h->sd.w = h->sd.z = nullptr;
    TRY(dalloc(h, &h->sd.w, (size_t)h->pl.n * (size_t)nrhs));
    TRY(dalloc(h, &h->sd.z, (size_t)h->pl.n * (size_t)nrhs));
    h->nrhs_cap = nrhs;
    return BASKER_OK;
}

// ---- precision 1: FP32 factorization, FP64 refinement

int ensure_twin(basker_t h)
{
    if (h->twin) return BASKER_OK;
    basker_options o = h->opt;
    o.precision = 0;
    return basker_symbolic(h->pl.n, h->in_colptr.data(), h->in_rowind.data(), h->in_P.data(), h->in_Q.data(),
                           h->in_nblocks, h->in_bptr.data(), h->in_ndblock, h->in_ndleaves,
                           h->in_ndptr.empty() ? nullptr : h->in_ndptr.data(), &o, &h->twin);
}

// FP64 factorization, by the twin, of the values of the last factorization call.
int factor_twin(basker_t h, cudaStream_t s)
{
    TRY(ensure_twin(h));
    const int st = h->twin->factored ? basker_refactor(h->twin, h->d_vals64, s)
                                     : basker_factor(h->twin, h->d_vals64, s);
    h->use64 = true;
    h->info.ir_fallbacks++;
    if (st != BASKER_OK) h->info.failed_column = h->twin->info.failed_column;
    return st;
}

// After the FP32 kernels: B in FP64 for the residual, ||B||_inf and the pivot
// growth; the FP64 twin takes over when the growth is too large or FP32 failed.
int finish_fp32(basker_t h, const double *values, cudaStream_t s, int st)
{
    h->use64 = false;
    h->fp32_valid = (st == BASKER_OK);
    if (st == BASKER_OK) {
        bk_launch_gather64(h->d, h->rf, values, h->pl.nnz, s);
        bk_launch_norms(h->d, h->rf, h->d_norms, s);
        CU(cudaMemcpyAsync(h->h_norms, h->d_norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        h->bnorm = h->h_norms[0];
        h->info.growth = h->h_norms[1];
        if (h->h_norms[1] <= h->opt.growth_limit) return BASKER_OK;   // false for NaN
    } else if (st != BASKER_ERR_SINGULAR && st != BASKER_ERR_NAN) {
        return st;
    }
    const int s64 = factor_twin(h, s);
    h->factored = (s64 == BASKER_OK);
    return s64;
}

// precision 2: FP64 factors; B in FP64 and ||B||_inf for the refined solves.
int finish_fp64(basker_t h, const double *values, cudaStream_t s)
{
    bk_launch_gather64(h->d, h->rf, values, h->pl.nnz, s);
    bk_launch_norms(h->d, h->rf, h->d_norms, s);
    CU(cudaMemcpyAsync(h->h_norms, h->d_norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    h->bnorm = h->h_norms[0];
    return BASKER_OK;
}

int ensure_ir_buffers(basker_t h, int32_t nrhs)
{
    if (nrhs <= h->ir_cap) return BASKER_OK;
    for (double **p : {&h->ir_c, &h->ir_r, &h->ir_z, &h->ir_dz, &h->d_irn}) {
        dfree(h, *p);
        *p = nullptr;
    }
    const size_t m = (size_t)h->pl.n * (size_t)nrhs;
    TRY(dalloc(h, &h->ir_c, m));
    TRY(dalloc(h, &h->ir_r, m));
    TRY(dalloc(h, &h->ir_z, m));
    TRY(dalloc(h, &h->ir_dz, m));
    TRY(dalloc(h, &h->d_irn, (size_t)3 * (size_t)nrhs));
    if (h->h_norms) cudaFreeHost(h->h_norms);
    h->h_norms = nullptr;
    CU(cudaMallocHost((void **)&h->h_norms, sizeof(double) * (2 + 3 * (size_t)nrhs)));
    h->ir_cap = nrhs;
    return BASKER_OK;
}

// x = A^{-1} b from the FP32 factors, refined in FP64 in B's space: z = 0,
// r = c = b(P); repeat dz = solve(r), z += dz, r = c - B z until the backward
// error reaches ir_tol.  A step that fails to halve it, or the last allowed
// step, hands the system to the FP64 twin.
int solve_refined(basker_t h, int32_t nrhs, const double *b, int32_t ldb, double *x, int32_t ldx, cudaStream_t s)
{
    if (h->use64) {
        h->info.precision_used = 0;
        h->info.ir_iterations = 0;
        return basker_solve(h->twin, nrhs, b, ldb, x, ldx, s);
    }
    TRY(ensure_ir_buffers(h, nrhs));
    TRY(ensure_solve_buffers(h, nrhs));
    const int32_t n = h->pl.n;
    double *cmax = h->d_irn, *zmax = cmax + nrhs, *rmax = zmax + nrhs;
    CU(cudaMemsetAsync(cmax, 0, sizeof(double) * (size_t)nrhs, s));
    tbeg(h, KT_REFINE, s, 1);
    bk_launch_ir_start(h->d, nrhs, b, ldb, h->ir_c, h->ir_r, h->ir_z, cmax, s);
    tend(h, s);
    double prev = INFINITY;
    for (int it = 1;; it++) {
        CU(cudaMemsetAsync(zmax, 0, sizeof(double) * 2 * (size_t)nrhs, s));
        CU(cudaMemsetAsync(h->d.counter + 2, 0, sizeof(int32_t), s));
        h->solve_epoch++;
        tbeg(h, KT_SOLVE, s, 1);
        bk_launch_solve(h->d, h->sd, nrhs, h->ir_r, n, h->ir_dz, n, h->solve_epoch, h->opt.wait_budget_cycles, s,
                        false, h->tune_solve);
        tend(h, s);
        tbeg(h, KT_REFINE, s, 2);
        bk_launch_ir_step(h->d, h->rf, nrhs, h->ir_c, h->ir_z, h->ir_dz, h->ir_r, zmax, rmax, s);
        tend(h, s);
        h->info.kernel_launches += 3;
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(h->h_norms + 2, cmax, sizeof(double) * 3 * (size_t)nrhs, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        double eta = 0.0;
        for (int32_t q = 0; q < nrhs; q++) {
            const double c = h->h_norms[2 + q], z = h->h_norms[2 + nrhs + q], r = h->h_norms[2 + 2 * nrhs + q];
            const double den = h->bnorm * z + c;
            const double e = den > 0.0 ? r / den : (r > 0.0 ? INFINITY : 0.0);
            eta = (e > eta || e != e) ? e : eta;
        }
        h->info.ir_iterations = it;
        h->info.ir_eta = eta;
        if (eta <= h->opt.ir_tol) break;
        if (h->opt.precision == 2 && (it >= h->opt.ir_max_iter || !(eta <= 0.5 * prev))) break;   // FP64 already
        if (it >= h->opt.ir_max_iter || !(eta <= 0.5 * prev)) {
            TRY(factor_twin(h, s));
            h->info.precision_used = 0;
            return basker_solve(h->twin, nrhs, b, ldb, x, ldx, s);
        }
        prev = eta;
    }
    bk_launch_ir_finish(h->d, nrhs, h->ir_z, x, ldx, s);
    h->info.precision_used = h->d.prec;
    CU(cudaGetLastError());
    return BASKER_OK;
}

}  // namespace

// Helpers of the allocation-free solve (noalloc.cu).  They launch the same solve
// kernel as basker_solve on scratch memory the caller provides and allocate
// nothing themselves.
int bk_handle_device(basker_t h) { return h ? h->device : -1; }

int32_t bk_handle_n(basker_t h) { return h->pl.n; }

int64_t bk_solve_scratch_doubles(basker_t h, int32_t nrhs)
{
    if (h->opt.precision) return INT64_MAX;    // the refinement needs buffers of its own
    return (int64_t)nrhs * 2 * (int64_t)h->pl.n;
}

int bk_solve_on_scratch(basker_t h, int32_t nrhs, const double *b_dev, int32_t ldb, double *x_dev, int32_t ldx,
                        double *scratch, void *stream)
{
    if (!h->factored) return BASKER_ERR_NOT_FACTORED;
    h->info.precision_used = 0;                // FP64 factors (refined handles are refused)
    if (nrhs == 0 || h->pl.n == 0) return BASKER_OK;
    bk_solve_dev sd = h->sd;
    sd.w = scratch;
    sd.z = scratch + (size_t)nrhs * (size_t)h->pl.n;
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemsetAsync(h->d.counter + 2, 0, sizeof(int32_t), s));
    h->solve_epoch++;
    h->info.kernel_launches++;
    bk_launch_solve(h->d, sd, nrhs, b_dev, ldb, x_dev, ldx, h->solve_epoch, h->opt.wait_budget_cycles, s, true,
                    h->tune_solve);
    CU(cudaGetLastError());
    return BASKER_OK;
}

extern "C" {

void basker_default_options(basker_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->tau = 1e-3;
    opt->slack = 1.0;
    opt->wait_budget_cycles = 20000000000LL;
    opt->factor_mode = 0;
    opt->precision = 0;
    opt->ir_max_iter = 10;
    opt->ir_tol = 1e-13;
    opt->growth_limit = 1e4;
    opt->graphs = 1;
}

const char *basker_strerror(int status)
{
    switch (status) {
    case BASKER_OK: return "ok";
    case BASKER_ERR_INVALID_ARG: return "invalid argument";
    case BASKER_ERR_NOT_BTF: return "matrix is not block upper triangular under P, Q";
    case BASKER_ERR_BAD_ND: return "an entry crosses an ND separator";
    case BASKER_ERR_SINGULAR: return "singular: no nonzero pivot candidate";
    case BASKER_ERR_NAN: return "non-finite value in a factored column";
    case BASKER_ERR_OOM: return "out of memory";
    case BASKER_ERR_TIMEOUT: return "in-kernel wait exceeded its budget";
    case BASKER_ERR_CUDA: return "CUDA runtime error";
    case BASKER_ERR_NOT_FACTORED: return "not factored";
    default: return "unknown status";
    }
}

int basker_symbolic_counts(int32_t n, const int32_t *colptr, const int32_t *rowind, const int32_t *P,
                           const int32_t *Q, int32_t nblocks, const int32_t *block_ptr, int32_t nd_block,
                           int32_t nd_leaves, const int32_t *nd_node_ptr, int mode, int32_t *l_count,
                           int32_t *u_count)
{
    if (mode < 0 || mode > 2) return BASKER_ERR_INVALID_ARG;
    bk_plan pl;
    int32_t bad = -1;
    const int st = bk_plan_build(n, colptr, rowind, P, Q, nblocks, block_ptr, nd_block, nd_leaves, nd_node_ptr,
                                 0.0, pl, &bad, mode);
    if (st != BASKER_OK) return st;
    if (l_count) std::copy(pl.sLcnt.begin(), pl.sLcnt.end(), l_count);
    if (u_count) std::copy(pl.sUcnt.begin(), pl.sUcnt.end(), u_count);
    return BASKER_OK;
}

int basker_symbolic(int32_t n, const int32_t *colptr, const int32_t *rowind, const int32_t *P,
                    const int32_t *Q, int32_t nblocks, const int32_t *block_ptr, int32_t nd_block,
                    int32_t nd_leaves, const int32_t *nd_node_ptr, const basker_options *opt,
                    basker_t *out)
{
    if (!out) return BASKER_ERR_INVALID_ARG;
    *out = nullptr;
    basker_t h = new (std::nothrow) basker_s();
    if (!h) return BASKER_ERR_OOM;
    basker_default_options(&h->opt);
    if (opt) h->opt = *opt;
    if (!(h->opt.tau > 0.0 && h->opt.tau <= 1.0) || h->opt.slack < 0.0 || h->opt.wait_budget_cycles <= 0 ||
        h->opt.factor_mode < 0 || h->opt.factor_mode > 1 || h->opt.precision < 0 || h->opt.precision > 2 ||
        h->opt.refactor_switch < 0 || h->opt.refactor_switch > 3 || h->opt.symbolic_mode < 0 ||
        h->opt.symbolic_mode > 2 ||
        (h->opt.precision >= 1 && (h->opt.ir_max_iter < 1 || !(h->opt.ir_tol > 0.0) || !(h->opt.growth_limit > 0.0)))) {
        delete h;
        return BASKER_ERR_INVALID_ARG;
    }
    cudaGetDevice(&h->device);
    if (h->opt.precision == 1 && n > 0 && colptr && rowind && P && Q && block_ptr && nblocks >= 0) {
        // kept to build the FP64 twin on first need
        h->in_colptr.assign(colptr, colptr + n + 1);
        h->in_rowind.assign(rowind, rowind + colptr[n]);
        h->in_P.assign(P, P + n);
        h->in_Q.assign(Q, Q + n);
        h->in_bptr.assign(block_ptr, block_ptr + nblocks + 1);
        if (nd_block >= 0 && nd_node_ptr) h->in_ndptr.assign(nd_node_ptr, nd_node_ptr + 2 * nd_leaves);
        h->in_nblocks = nblocks;
        h->in_ndblock = nd_block;
        h->in_ndleaves = nd_leaves;
    }
    int32_t bad = -1;
    int st = bk_plan_build(n, colptr, rowind, P, Q, nblocks, block_ptr, nd_block, nd_leaves, nd_node_ptr,
                           h->opt.slack, h->pl, &bad, h->opt.symbolic_mode);
    if (st == BASKER_OK) st = setup_device(h);
    if (st != BASKER_OK) {
        h->info.failed_column = bad;
        basker_free(h);
        return st;
    }
    h->info.n = n;
    h->info.nblocks = nblocks;
    h->info.nd_block = h->pl.nd_block;
    h->info.nd_leaves = h->pl.nd_leaves;
    h->info.nnz_a = h->pl.nnz;
    h->info.nnz_l_sym = h->pl.nnz_l_sym;
    h->info.nnz_u_sym = h->pl.nnz_u_sym;
    h->info.failed_column = -1;
    *out = h;
    return BASKER_OK;
}

int basker_factor(basker_t h, const double *values_dev, void *stream)
{
    if (!h || (!values_dev && h->pl.nnz > 0)) return BASKER_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    h->factored = false;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opt.precision && h->pl.nnz > 0)
        CU(cudaMemcpyAsync(h->d_vals64, values_dev, sizeof(double) * (size_t)h->pl.nnz, cudaMemcpyDeviceToDevice, s));
    int st = factor_impl(h, values_dev, s, false);
    h->info.gp_launches = h->launches;
    if (h->opt.precision == 1) st = finish_fp32(h, values_dev, s, st);
    if (h->opt.precision == 2 && st == BASKER_OK) st = finish_fp64(h, values_dev, s);
    return st;
}

int basker_refactor(basker_t h, const double *values_dev, void *stream)
{
    if (!h || (!values_dev && h->pl.nnz > 0)) return BASKER_ERR_INVALID_ARG;
    if (!h->factored) return BASKER_ERR_NOT_FACTORED;
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opt.precision && h->pl.nnz > 0)
        CU(cudaMemcpyAsync(h->d_vals64, values_dev, sizeof(double) * (size_t)h->pl.nnz, cudaMemcpyDeviceToDevice, s));
    // FP32 factors that failed last time are not a base to refactor from
    const bool re = h->opt.precision != 1 || h->fp32_valid;
    if (!re) h->factored = false;
    int st = factor_impl(h, values_dev, s, re);
    h->info.static_launches = h->launches;
    if (h->opt.precision == 1) st = finish_fp32(h, values_dev, s, st);
    if (h->opt.precision == 2 && st == BASKER_OK) st = finish_fp64(h, values_dev, s);
    return st;
}

int basker_solve(basker_t h, int32_t nrhs, const double *b_dev, int32_t ldb, double *x_dev, int32_t ldx,
                 void *stream)
{
    if (!h || nrhs < 0 || (nrhs > 0 && (!b_dev || !x_dev || ldb < h->pl.n || ldx < h->pl.n)))
        return BASKER_ERR_INVALID_ARG;
    if (!h->factored) return BASKER_ERR_NOT_FACTORED;
    if (nrhs == 0 || h->pl.n == 0) return BASKER_OK;
    cudaSetDevice(h->device);
    if (h->opt.precision) return solve_refined(h, nrhs, b_dev, ldb, x_dev, ldx, (cudaStream_t)stream);
    TRY(ensure_solve_buffers(h, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaMemsetAsync(h->d.counter + 2, 0, sizeof(int32_t), s));
    h->solve_epoch++;
    h->info.precision_used = 0;
    tbeg(h, KT_SOLVE, s, 1);
    bk_launch_solve(h->d, h->sd, nrhs, b_dev, ldb, x_dev, ldx, h->solve_epoch, h->opt.wait_budget_cycles, s, true,
                    h->tune_solve);
    tend(h, s);
    CU(cudaGetLastError());
    return BASKER_OK;
}

int basker_refactor_solve_host(basker_t h, const double *values_host, int32_t nrhs, const double *b_host,
                               double *x_host, void *stream)
{
    if (!h || !values_host || nrhs < 0 || (nrhs > 0 && (!b_host || !x_host))) return BASKER_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)h->pl.n;
    if (!h->d_vals) TRY(dalloc(h, &h->d_vals, (size_t)h->pl.nnz));
    if (nrhs > h->stage_nrhs) {
        dfree(h, h->d_b);
        dfree(h, h->d_x);
        h->d_b = h->d_x = nullptr;
        TRY(dalloc(h, &h->d_b, n * (size_t)nrhs));
        TRY(dalloc(h, &h->d_x, n * (size_t)nrhs));
        h->stage_nrhs = nrhs;
    }
    CU(cudaMemcpyAsync(h->d_vals, values_host, sizeof(double) * (size_t)h->pl.nnz, cudaMemcpyHostToDevice, s));
    if (nrhs > 0) CU(cudaMemcpyAsync(h->d_b, b_host, sizeof(double) * n * (size_t)nrhs, cudaMemcpyHostToDevice, s));
    int st = h->factored ? basker_refactor(h, h->d_vals, stream) : basker_factor(h, h->d_vals, stream);
    if (st != BASKER_OK) return st;
    if (nrhs > 0) {
        TRY(basker_solve(h, nrhs, h->d_b, (int32_t)n, h->d_x, (int32_t)n, stream));
        CU(cudaMemcpyAsync(x_host, h->d_x, sizeof(double) * n * (size_t)nrhs, cudaMemcpyDeviceToHost, s));
    }
    CU(cudaStreamSynchronize(s));
    return BASKER_OK;
}

int basker_info(basker_t h, basker_info_t *out)
{
    if (!h || !out) return BASKER_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    h->info.device_bytes = h->device_bytes;
    h->info.cuda_error = g_cuda_err;
    h->info.cuda_line = g_cuda_line;
    tflush(h);
    *out = h->info;
    for (double &v : h->info.kernel_ms) v = 0.0;
    for (int32_t &v : h->info.kernel_calls) v = 0;
    h->info.rounds_columns = 0;
    if (!h->factored) return BASKER_OK;
    {
        const size_t n = (size_t)h->pl.n;
        std::vector<int32_t> lc(n), uc(n);
        CU(device_sync());
        CU(cudaMemcpy(lc.data(), h->d.Lcnt, n * 4, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(uc.data(), h->d.Ucnt, n * 4, cudaMemcpyDeviceToHost));
        int64_t nl = 0, nu = 0;
        for (size_t c = 0; c < n; c++) { nl += lc[c]; nu += uc[c]; }
        h->info.nnz_l = nl;
        h->info.nnz_u = nu;
        // flops: sum_j l_j (2 u_j + 1), u_j = entries right of the diagonal in row j
        // of U, from the row starts of the factors by rows (rebuilt after every
        // factorization)
        std::vector<int64_t> urp(n + 1);
        CU(cudaMemcpy(urp.data(), h->sd.r.Urp, (n + 1) * 8, cudaMemcpyDeviceToHost));
        double fl = 0;
        for (size_t c = 0; c < n; c++) fl += (double)lc[c] * (2.0 * (double)(urp[c + 1] - urp[c]) + 1.0);
        h->info.flops = fl;
        std::vector<int32_t> pr(n);
        CU(cudaMemcpy(pr.data(), h->d.prow, n * 4, cudaMemcpyDeviceToHost));
        int32_t off = 0;
        for (size_t c = 0; c < n; c++) off += pr[c] != (int32_t)c;
        h->info.off_diagonal_pivots = off;
        out->nnz_l = nl;
        out->nnz_u = nu;
        out->flops = fl;
        out->off_diagonal_pivots = off;
    }
    return BASKER_OK;
}

int basker_export(basker_t h, int32_t *prow, int64_t *Lp, int32_t *Li, double *Lx, int64_t *Up, int32_t *Ui,
                  double *Ux, int64_t *nnz_l, int64_t *nnz_u)
{
    if (!h || !nnz_l || !nnz_u) return BASKER_ERR_INVALID_ARG;
    if (!h->factored) return BASKER_ERR_NOT_FACTORED;
    cudaSetDevice(h->device);
    CU(device_sync());
    const size_t n = (size_t)h->pl.n;
    std::vector<int32_t> lc(n), uc(n), pr(n), pinv(n);
    std::vector<int64_t> lb(n + 1), ub(n + 1);
    CU(cudaMemcpy(lc.data(), h->d.Lcnt, n * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(uc.data(), h->d.Ucnt, n * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(pr.data(), h->d.prow, n * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(pinv.data(), h->d.pinv, n * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(lb.data(), h->d.Lbeg, (n + 1) * 8, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(ub.data(), h->d.Ubeg, (n + 1) * 8, cudaMemcpyDeviceToHost));
    int64_t nl = 0, nu = 0;
    for (size_t c = 0; c < n; c++) { nl += lc[c]; nu += uc[c]; }
    *nnz_l = nl;
    *nnz_u = nu;
    if (!Li) return BASKER_OK;
    if (!prow || !Lp || !Lx || !Up || !Ui || !Ux) return BASKER_ERR_INVALID_ARG;
    std::vector<int32_t> li((size_t)h->d.lpool_end), ui((size_t)h->d.upool_end);
    std::vector<double> lx((size_t)h->d.lpool_end), ux((size_t)h->d.upool_end);
    CU(cudaMemcpy(li.data(), h->d.Li, li.size() * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(ui.data(), h->d.Ui, ui.size() * 4, cudaMemcpyDeviceToHost));
    if (h->d.prec) {
        // FP32 factors, widened
        std::vector<float> f(std::max(lx.size(), ux.size()));
        CU(cudaMemcpy(f.data(), h->d.Lx, lx.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < lx.size(); i++) lx[i] = f[i];
        CU(cudaMemcpy(f.data(), h->d.Ux, ux.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < ux.size(); i++) ux[i] = f[i];
    } else {
        CU(cudaMemcpy(lx.data(), h->d.Lx, lx.size() * 8, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(ux.data(), h->d.Ux, ux.size() * 8, cudaMemcpyDeviceToHost));
    }
    std::memcpy(prow, pr.data(), n * 4);
    Lp[0] = Up[0] = 0;
    std::vector<std::pair<int32_t, double>> col;
    for (size_t c = 0; c < n; c++) {
        col.clear();
        for (int32_t k = 0; k < lc[c]; k++) {
            const int32_t r = li[(size_t)(lb[c] + k)];
            col.emplace_back(r >= 0 && (size_t)r < n ? pinv[(size_t)r] : -1, lx[(size_t)(lb[c] + k)]);
        }
        std::sort(col.begin(), col.end(), [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
            return a.first < b.first;
        });
        int64_t o = Lp[c];
        for (auto &e : col) { Li[o] = e.first; Lx[o] = e.second; o++; }
        Lp[c + 1] = o;
        int64_t q = Up[c];
        for (int32_t k = 0; k < uc[c]; k++) {
            Ui[q] = ui[(size_t)(ub[c] + k)];
            Ux[q] = ux[(size_t)(ub[c] + k)];
            q++;
        }
        Up[c + 1] = q;
    }
    return BASKER_OK;
}

int basker_autotune(basker_t h, const double *values_dev, const double *b_dev, void *stream)
{
    if (!h || (!values_dev && h->pl.nnz > 0) || (!b_dev && h->pl.n > 0)) return BASKER_ERR_INVALID_ARG;
    if (!h->factored) return BASKER_ERR_NOT_FACTORED;
    if (h->pl.n == 0) return BASKER_OK;
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n = h->pl.n;
    double *x = nullptr;
    TRY(dalloc(h, &x, (size_t)n));
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    sms = std::max(sms, 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    int st = BASKER_OK;
    // one trial: the best of two refactor + solve runs
    auto trial = [&]() -> float {
        float best = 1e30f;
        for (int rep = 0; rep < 2 && st == BASKER_OK; rep++) {
            cudaEventRecord(e0, s);
            st = basker_refactor(h, values_dev, s);
            if (st == BASKER_OK) st = basker_solve(h, 1, b_dev, n, x, n, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = BASKER_ERR_CUDA;
            float ms = 0.f;
            if (st == BASKER_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, ms);
        }
        return best;
    };
    // coordinate search: the stored-pattern pass's persistent blocks per SM (up to
    // the allocated per-warp slices), then the solve's, then the rounds' warps
    auto search = [&](int &knob, const std::vector<int> &cands) {
        float bt = 1e30f;
        int bk = 0;
        for (int v : cands) {
            knob = v;
            const float t = trial();
            if (st != BASKER_OK) return;
            if (t < bt) { bt = t; bk = v; }
        }
        knob = bk;
    };
    std::vector<int> cs, cv, cd;
    for (int per = 1; per * sms <= bk_static_blocks(); per++) cs.push_back(per * sms);
    for (int per = 2; per * sms <= bk_solve_blocks(); per += 2) cv.push_back(per * sms);
    for (int w = h->pl.wsd_warps; w >= 152 && cd.size() < 3; w /= 2) cd.push_back(w);
    search(h->tune_static, cs);
    if (st == BASKER_OK) search(h->tune_solve, cv);
    if (st == BASKER_OK) search(h->tune_dd, cd);
    if (st != BASKER_OK) h->tune_static = h->tune_solve = h->tune_dd = 0;
    h->info.tuned_static_blocks = h->tune_static;
    h->info.tuned_solve_blocks = h->tune_solve;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(h, x);
    return st;
}

#ifdef BK_TRACE
// Diagnostic builds only: copy out the per-item timeline (4 words a record, see
// trace.cuh) recorded since the last call, then restart it.
int basker_trace_read(basker_t h, unsigned long long *host, int64_t max_records, int64_t *count)
{
    if (!h || !h->d.trace || !count) return BASKER_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    CU(cudaDeviceSynchronize());
    unsigned long long total = 0;
    CU(cudaMemcpy(&total, h->d.trace, sizeof(total), cudaMemcpyDeviceToHost));
    const int64_t m = std::min<int64_t>(std::min<int64_t>((int64_t)total, BK_TRACE_CAP), max_records);
    if (host && m > 0) CU(cudaMemcpy(host, h->d.trace + 4, (size_t)m * 32, cudaMemcpyDeviceToHost));
    *count = (int64_t)total;
    CU(cudaMemset(h->d.trace, 0, sizeof(total)));
    return BASKER_OK;
}
#endif

void basker_free(basker_t h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    {
        std::lock_guard<std::mutex> lk(g_capture_mu);
        cudaDeviceSynchronize();
        for (auto &a : h->allocs) cudaFree(a.first);
    }
    if (h->h_stage) cudaFreeHost(h->h_stage);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->h_task_fail) cudaFreeHost(h->h_task_fail);
    for (auto &t : h->pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    if (h->open_ev) cudaEventDestroy(h->open_ev);
    if (h->h_norms) cudaFreeHost(h->h_norms);
    if (h->twin) basker_free(h->twin);
    if (h->g_finish) cudaGraphExecDestroy(h->g_finish);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

}  // extern "C"
