// nl_batch.cu -- many uneven 2-D instances (each its own grid, horizon and coefficient
// fields) applied in one persistent launch, and solved together by CG.
//
// The batch owns one plan per instance.  Its fields are concatenated instance by instance
// (instance k occupies elements offsets[k] .. offsets[k+1]-1 of every vector; peridynamic
// instances hold their two component planes there).  The apply is one launch of a persistent
// kernel whose blocks pull (instance, tile) work items from an atomic counter.  The tile shape
// is 32 x 4, 32 x 8 or 32 x 16 threads; nl_batch_create can time the three on the batch and
// keep the fastest (the autotuner, tile_shape = NL_TILE_AUTO).  CG treats each instance as one right-hand side segment,
// so all instances iterate together in one captured graph.
#include <cstdlib>
#include <cstring>
#include <vector>

#include "nl_internal.cuh"

#define NL_BATCH_MAGIC 0x4e4c4254u   // "NLBT"

enum { BK_SCALAR = 0, BK_SYM = 1, BK_PD = 2, BK_PDX2 = 3 };

struct nl_batch {
    uint32_t magic;
    const double *skip;           // CG convergence flags while a batched CG runs, else null
    int skip_stride;
    int count, kind, kind32, Rmax, shape;   // kind32: kernel of FP32 applies
    int all_symmetric;
    nl_plan **plans;
    int64_t *off;                 // host [count + 1]
    int64_t *seg_off, *seg_len;   // device [count]
    void *inst[2];                // device instance tables for FP32 and FP64
    int64_t total_tiles[2];       // FP32 and FP64 tables
    int *counter;
    nl_cg_state cg;
};

static bool batch_ok(const nl_batch *b) { return b && b->magic == NL_BATCH_MAGIC; }

static nl_status build_tables(nl_batch *b, int shape, cudaStream_t st)
{
    const size_t bytes = nl_batch_inst_bytes() * b->count;
    std::vector<unsigned char> host(bytes);
    for (int t = 0; t < 2; ++t) {
        int64_t total = 0;
        nl_batch_fill_inst(b->plans, b->count, b->off, shape, t == 0 ? NL_F32 : NL_F64,
                           t == 0 ? b->kind32 : b->kind, host.data(), &total);
        b->total_tiles[t] = total;
        if (!b->inst[t]) {
            if (cudaMalloc(&b->inst[t], bytes) != cudaSuccess) {
                nl_set_error("nl_batch_create: device allocation failed");
                return NL_ENOMEM;
            }
        }
        NL_CUDA_TRY(cudaMemcpyAsync(b->inst[t], host.data(), bytes, cudaMemcpyHostToDevice, st));
        NL_CUDA_TRY(cudaStreamSynchronize(st));
    }
    b->shape = shape;
    return NL_OK;
}

static nl_status batch_launch(nl_batch *b, const void *u, void *Lu, int dtype, cudaStream_t st)
{
    const int t = dtype == NL_F32 ? 0 : 1;
    return nl_batch_launch(t == 0 ? b->kind32 : b->kind, b->shape, dtype, b->inst[t], b->count,
                           b->total_tiles[t], b->counter, u, Lu, b->Rmax, st);
}

extern "C" nl_status nl_batch_destroy(nl_batch *b)
{
    if (!b) return NL_OK;
    if (!batch_ok(b)) {
        nl_set_error("nl_batch_destroy: not a batch");
        return NL_EINVAL;
    }
    cudaDeviceSynchronize();
    for (int k = 0; k < b->count; ++k)
        if (b->plans && b->plans[k]) nl_plan_destroy(b->plans[k]);
    free(b->plans);
    free(b->off);
    void *ptrs[] = { b->seg_off, b->seg_len, b->inst[0], b->inst[1], b->counter };
    for (void *q : ptrs) if (q) cudaFree(q);
    nl_cg_state_release(&b->cg);
    b->magic = 0;
    free(b);
    return NL_OK;
}

extern "C" nl_status nl_batch_create(nl_batch **out, int count, const nl_grid *grids,
                                     const nl_horizon *horizons, const nl_kernel *kernels,
                                     int tile_shape, void *stream)
{
    if (!out || count < 1 || count > 65535 || !grids || !horizons || !kernels ||
        tile_shape < NL_TILE_AUTO || tile_shape > NL_TILE_32x16) {
        nl_set_error("nl_batch_create: bad argument");
        return NL_EINVAL;
    }
    *out = nullptr;
    for (int k = 0; k < count; ++k) {
        if (grids[k].dim != 2 || (kernels[k].family != NL_POWER && kernels[k].family != NL_PD_BOND) ||
            kernels[k].family != kernels[0].family || !!horizons[k].symmetric != !!horizons[0].symmetric) {
            nl_set_error("nl_batch_create: instances must be 2-D and share the family (NL_POWER "
                         "or NL_PD_BOND) and the symmetric flag (instance %d differs)", k);
            return NL_EUNSUPPORTED;
        }
    }
    cudaStream_t st = nl_stream(stream);
    nl_batch *b = (nl_batch *)calloc(1, sizeof(nl_batch));
    if (!b) return NL_ENOMEM;
    b->magic = NL_BATCH_MAGIC;
    b->count = count;
    b->plans = (nl_plan **)calloc(count, sizeof(nl_plan *));
    b->off = (int64_t *)calloc(count + 1, sizeof(int64_t));
    if (!b->plans || !b->off) { nl_batch_destroy(b); return NL_ENOMEM; }
    const bool pd = kernels[0].family == NL_PD_BOND;
    b->kind = pd ? BK_PD : (horizons[0].symmetric ? BK_SYM : BK_SCALAR);
    b->all_symmetric = 1;
    for (int k = 0; k < count; ++k) {
        nl_status s = nl_plan_create(&b->plans[k], &grids[k], &horizons[k], &kernels[k], stream);
        if (s != NL_OK) { nl_batch_destroy(b); return s; }
        const nl_plan *p = b->plans[k];
        b->Rmax = p->Rmax > b->Rmax ? p->Rmax : b->Rmax;
        b->off[k + 1] = b->off[k] + (pd ? 2 : 1) * p->N;
        if (!(p->symmetric || (pd && p->const_horizon))) b->all_symmetric = 0;
    }
    // FP32 peridynamic applies take the paired-column kernel when every horizon is constant
    b->kind32 = b->kind;
    if (pd && b->Rmax <= 32) {
        bool x2 = true;
        for (int k = 0; k < count && x2; ++k) x2 = b->plans[k]->pd_dense32 != nullptr;
        if (x2) b->kind32 = BK_PDX2;
    }
    std::vector<int64_t> so(count), sl(count);
    for (int k = 0; k < count; ++k) { so[k] = b->off[k]; sl[k] = b->off[k + 1] - b->off[k]; }
    if (cudaMalloc(&b->seg_off, count * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->seg_len, count * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&b->counter, sizeof(int)) != cudaSuccess) {
        nl_batch_destroy(b);
        nl_set_error("nl_batch_create: device allocation failed");
        return NL_ENOMEM;
    }
    cudaError_t ce = cudaMemcpyAsync(b->seg_off, so.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(b->seg_len, sl.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) { nl_batch_destroy(b); return nl_cuda_fail(ce, "nl_batch_create upload"); }
    nl_status s = build_tables(b, tile_shape == NL_TILE_AUTO ? NL_TILE_32x8 : tile_shape, st);
    if (s != NL_OK) { nl_batch_destroy(b); return s; }
    if (tile_shape == NL_TILE_AUTO) {
        // time each tile shape on the batch (FP32, zero input) and keep the fastest
        const int64_t len = b->off[count];
        float *u = nullptr, *lu = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaMalloc(&u, len * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&lu, len * sizeof(float)) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (u) cudaFree(u);
            if (lu) cudaFree(lu);
            nl_batch_destroy(b);
            nl_set_error("nl_batch_create: autotune allocation failed");
            return NL_ENOMEM;
        }
        cudaMemsetAsync(u, 0, len * sizeof(float), st);
        float best = 1e30f;
        int best_shape = 1;
        for (int shape = 0; shape < 3 && s == NL_OK; ++shape) {
            if ((s = build_tables(b, shape, st)) != NL_OK) break;
            if ((s = batch_launch(b, u, lu, NL_F32, st)) != NL_OK) {
                if (s == NL_EUNSUPPORTED) { s = NL_OK; continue; }   // tile too large
                break;
            }
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && s == NL_OK; ++r) s = batch_launch(b, u, lu, NL_F32, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (s == NL_OK && ms < best) { best = ms; best_shape = shape; }
        }
        cudaFree(u);
        cudaFree(lu);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s == NL_OK) s = build_tables(b, best_shape, st);
        if (s != NL_OK) { nl_batch_destroy(b); return s; }
    }
    *out = b;
    return NL_OK;
}

extern "C" nl_status nl_batch_layout(const nl_batch *b, int64_t *offsets, int *tile_shape)
{
    if (!batch_ok(b) || !offsets) {
        nl_set_error("nl_batch_layout: bad argument");
        return NL_EINVAL;
    }
    memcpy(offsets, b->off, (b->count + 1) * sizeof(int64_t));
    if (tile_shape) *tile_shape = b->shape;
    return NL_OK;
}

extern "C" nl_status nl_batch_apply(nl_batch *b, const void *u, void *Lu, int dtype, void *stream)
{
    if (!batch_ok(b) || !u || !Lu || (dtype != NL_F32 && dtype != NL_F64)) {
        nl_set_error("nl_batch_apply: bad argument");
        return NL_EINVAL;
    }
    return batch_launch(b, u, Lu, dtype, nl_stream(stream));
}

struct BatchOpCtx { nl_batch *b; };

static nl_status bop_apply(void *ctx, const void *in, void *out, int dtype, cudaStream_t st)
{
    nl_batch *b = ((BatchOpCtx *)ctx)->b;
    if (dtype != NL_F32 || !b->skip) return batch_launch(b, in, out, dtype, st);
    // inside the iterations (FP32): converged instances are skipped
    return nl_batch_launch(b->kind32, b->shape, dtype, b->inst[0], b->count, b->total_tiles[0],
                           b->counter, in, out, b->Rmax, st, b->skip, b->skip_stride);
}

static void bop_set_skip(void *ctx, const double *flags, int stride)
{
    nl_batch *b = ((BatchOpCtx *)ctx)->b;
    b->skip = flags;
    b->skip_stride = stride;
}

static nl_status bop_diag(void *ctx, const double *zin, double *d, cudaStream_t st)
{
    nl_batch *b = ((BatchOpCtx *)ctx)->b;
    for (int k = 0; k < b->count; ++k) {
        nl_status s = nl_diag_launch(b->plans[k], zin + b->off[k], d + b->off[k], st);
        if (s != NL_OK) return s;
    }
    return NL_OK;
}

extern "C" nl_status nl_batch_cg_solve(nl_batch *b, const void *f, void *x, double rtol,
                                       int maxit, int precond, nl_cg_stats *stats, void *stream)
{
    if (!batch_ok(b)) {
        nl_set_error("nl_batch_cg_solve: invalid batch");
        return NL_EINVAL;
    }
    if (!b->all_symmetric || precond == NL_PRECOND_LEARNED) {
        nl_set_error("nl_batch_cg_solve: needs symmetric instances (symmetric NL_POWER, or "
                     "NL_PD_BOND with constant horizons) and Jacobi or no preconditioner");
        return NL_EUNSUPPORTED;
    }
    BatchOpCtx ctx{ b };
    nl_cg_op op;
    memset(&op, 0, sizeof(op));
    op.nrhs = b->count;
    op.per = 0;
    op.total = b->off[b->count];
    op.seg_off = b->seg_off;
    op.seg_len = b->seg_len;
    op.dinv_len = op.total;
    op.apply = bop_apply;
    op.diag = bop_diag;
    op.set_skip = bop_set_skip;
    op.ctx = &ctx;
    op.state = &b->cg;
    const nl_status s = nl_cg_run(op, f, x, rtol, maxit, precond, nullptr, 0, nullptr, stats, stream);
    bop_set_skip(&ctx, nullptr, 0);
    return s;
}
