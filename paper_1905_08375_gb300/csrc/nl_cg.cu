// nl_cg.cu -- preconditioned conjugate gradients on -L x = f, the Krylov use of the fast
// matrix-vector product remarked in the paper's conclusion (Sec. 4).
//
// Precision: x, r, z, p and every inner product are FP64; the operator is applied in FP32
// to an FP32 copy of p (written by the direction update), and its FP32 result enters the
// FP64 updates.  When the recursive residual of every right-hand side is below the
// tolerance, the true residual f + L x is recomputed with the FP64 operator (on 2-D
// symmetric NL_POWER plans its FP32-pair form, NL_F64_PAIRS); right-hand
// sides that miss the tolerance restart from that true residual (defect correction), so
// the reported residual is always the FP64 one.
//
// Execution: per right-hand side, nb <= NB blocks do grid-stride vector work and write one
// partial sum each (nb = NB for one right-hand side or uneven segments, fewer per right-hand
// side when several share the grid); the next kernel folds the nb partials in a fixed order
// (same value in
// every block, deterministic).  One iteration is four launches (apply, dot, update,
// direction); CHUNK iterations plus a convergence check are captured once into a CUDA
// graph on a plan-owned stream.  The host reads the per-right-hand-side flags from pinned
// memory after each chunk, with a bounded wait.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <cmath>
#include <thread>

#include "nl_internal.cuh"

namespace {

constexpr int RB = 256;     // threads per reduction block
constexpr int NB = 152;     // reduction blocks per right-hand side at most (one per SM)
constexpr int CG_GRID_WAVES = 2;   // uniform segments: about CG_GRID_WAVES x NB blocks in all
constexpr int CHUNK = 16;   // iterations per captured graph
constexpr int CHUNK_TAIL = 4;   // iterations per graph once convergence is predicted within CHUNK

// per right-hand side scalars
enum { S_RZ = 0, S_FF, S_RR, S_CONV, S_IT, S_TRUE, S_COUNT = 8 };
// partial-sum slots
enum { P_PQ = 0, P_RZ, P_RR, P_AUX, P_COUNT };

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < RB / 32) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;   // valid in thread 0
}

// sum of the nb partials of (slot, rhs), fixed order; valid in every lane of warp 0
__device__ __forceinline__ double fold(const double *part, int slot, int rhs, int nrhs, int nb)
{
    const double *q = part + ((size_t)slot * nrhs + rhs) * NB;
    double s = 0.0;
    for (int k = threadIdx.x & 31; k < nb; k += 32) s += q[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

struct CgArgs {
    int64_t per;          // unknowns per right-hand side (uniform segments)
    const int64_t *seg_off, *seg_len;   // per-segment offsets/lengths, or nullptr
    int dinv_global;      // dinv indexed by the global position (else by k)
    int nrhs;
    int nb;               // blocks per right-hand side (<= NB)
    double tol;           // on the recursive relative residual
    const double *f;
    double *x, *r, *z, *p, *q64;
    const double *dinv;   // [per]
    float *p32, *q32;
    double *part;         // [P_COUNT][nrhs][NB]
    double *sc;           // [nrhs][S_COUNT]
};

__device__ __forceinline__ int64_t seg_base(const CgArgs &a, int rhs)
{
    return a.seg_off ? a.seg_off[rhs] : (int64_t)rhs * a.per;
}
__device__ __forceinline__ int64_t seg_len(const CgArgs &a, int rhs)
{
    return a.seg_len ? a.seg_len[rhs] : a.per;
}
__device__ __forceinline__ double dinv_at(const CgArgs &a, int64_t base, int64_t k)
{
    return a.dinv[a.dinv_global ? base + k : k];
}

__device__ __forceinline__ void store_partial(const CgArgs &a, int slot, int rhs, double v)
{
    a.part[((size_t)slot * a.nrhs + rhs) * NB + blockIdx.x] = v;
}

// r = f, x = 0; z = D^{-1} r and p = z unless FLEX (the network computes z afterwards)
template <bool FLEX>
__global__ void __launch_bounds__(RB) k_cg_init(CgArgs a)
{
    __shared__ double sh[RB / 32];
    const int rhs = blockIdx.y;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double rz = 0.0, rr = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB) {
        const double fv = a.f[base + k];
        a.x[base + k] = 0.0;
        a.r[base + k] = fv;
        if (!FLEX) {
            const double zv = dinv_at(a, base, k) * fv;
            a.z[base + k] = zv;
            a.p[base + k] = zv;
            a.p32[base + k] = (float)zv;
            rz += fv * zv;
        }
        rr += fv * fv;
    }
    double s;
    s = block_sum(rz, sh); if (threadIdx.x == 0) store_partial(a, P_RZ, rhs, s);
    s = block_sum(rr, sh); if (threadIdx.x == 0) { store_partial(a, P_RR, rhs, s); store_partial(a, P_AUX, rhs, s); }
}

__global__ void k_cg_init_scalars(CgArgs a)
{
    const int rhs = blockIdx.x;
    if (threadIdx.x >= 32) return;
    const double ff = fold(a.part, P_AUX, rhs, a.nrhs, a.nb);
    if (threadIdx.x == 0) {
        double *sc = a.sc + (size_t)rhs * S_COUNT;
        sc[S_FF] = ff;
        sc[S_CONV] = (ff == 0.0) ? 1.0 : 0.0;
        sc[S_IT] = 0.0;
        sc[S_TRUE] = 0.0;
    }
}

// FLEX: after the network wrote z = M(r): for right-hand sides selected by `only`
// (all when only < 0; else those with sc[S_TRUE] > goal) set p = z; partial r.z
__global__ void __launch_bounds__(RB) k_cg_pz(CgArgs a, int only, double goal)
{
    __shared__ double sh[RB / 32];
    const int rhs = blockIdx.y;
    const bool redo = only < 0 || a.sc[(size_t)rhs * S_COUNT + S_TRUE] > goal;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double rz = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB) {
        const int64_t g = base + k;
        const double zv = a.z[g];
        if (redo) {
            a.p[g] = zv;
            a.p32[g] = (float)zv;
        }
        rz += a.r[g] * zv;
    }
    const double s = block_sum(rz, sh);
    if (threadIdx.x == 0) store_partial(a, P_RZ, rhs, s);
}

// Folds the r.z and r.r partials of the last update into rz_old and the convergence flag.
// Idempotent: repeating it without an update in between changes nothing.
__device__ __forceinline__ void scalars_after_update(const CgArgs &a, int rhs)
{
    const double rz = fold(a.part, P_RZ, rhs, a.nrhs, a.nb);
    const double rr = fold(a.part, P_RR, rhs, a.nrhs, a.nb);
    if (threadIdx.x == 0) {
        double *sc = a.sc + (size_t)rhs * S_COUNT;
        sc[S_RZ] = rz;
        sc[S_RR] = rr;
        if (sc[S_CONV] == 0.0 && rr <= a.tol * a.tol * sc[S_FF]) sc[S_CONV] = 1.0;
    }
}

__global__ void k_cg_check(CgArgs a)
{
    if (threadIdx.x < 32) scalars_after_update(a, blockIdx.x);
}

// partial (p, A p) with A p = -q (q = L p in FP32)
__global__ void __launch_bounds__(RB) k_cg_dot(CgArgs a)
{
    __shared__ double sh[RB / 32];
    const int rhs = blockIdx.y;
    if (blockIdx.x == 0 && threadIdx.x < 32) scalars_after_update(a, rhs);
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double pq = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB)
        pq -= a.p[base + k] * (double)a.q32[base + k];
    const double s = block_sum(pq, sh);
    if (threadIdx.x == 0) store_partial(a, P_PQ, rhs, s);
}

// x += alpha p, r -= alpha A p; then z = D^{-1} r with partial r.z, or (FLEX) partial
// r_new . z_old for the flexible beta; partial r.r either way
template <bool FLEX>
__global__ void __launch_bounds__(RB) k_cg_update(CgArgs a)
{
    __shared__ double sh[RB / 32];
    __shared__ double s_alpha;
    const int rhs = blockIdx.y;
    const double *sc = a.sc + (size_t)rhs * S_COUNT;
    if (threadIdx.x < 32) {
        const double pq = fold(a.part, P_PQ, rhs, a.nrhs, a.nb);
        if (threadIdx.x == 0) {
            const bool live = sc[S_CONV] == 0.0 && pq > 0.0 && sc[S_RZ] > 0.0;
            s_alpha = live ? sc[S_RZ] / pq : 0.0;
            if (live && blockIdx.x == 0) a.sc[(size_t)rhs * S_COUNT + S_IT] += 1.0;
        }
    }
    __syncthreads();
    const double alpha = s_alpha;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double rz = 0.0, rr = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB) {
        const int64_t g = base + k;
        double rv = a.r[g];
        if (alpha != 0.0) {
            a.x[g] += alpha * a.p[g];
            rv += alpha * (double)a.q32[g];
            a.r[g] = rv;
        }
        if (FLEX) {
            rz += rv * a.z[g];
        } else {
            const double zv = dinv_at(a, base, k) * rv;
            a.z[g] = zv;
            rz += rv * zv;
        }
        rr += rv * rv;
    }
    double s;
    s = block_sum(rz, sh); if (threadIdx.x == 0) store_partial(a, FLEX ? P_AUX : P_RZ, rhs, s);
    s = block_sum(rr, sh); if (threadIdx.x == 0) store_partial(a, P_RR, rhs, s);
}

// FLEX: partial r.z after the network wrote the new z
__global__ void __launch_bounds__(RB) k_cg_rz(CgArgs a)
{
    __shared__ double sh[RB / 32];
    const int rhs = blockIdx.y;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double rz = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB)
        rz += a.r[base + k] * a.z[base + k];
    const double s = block_sum(rz, sh);
    if (threadIdx.x == 0) store_partial(a, P_RZ, rhs, s);
}

// p = z + beta p, p32 = (float) p.  beta = r+.z+ / r.z, or for the flexible method
// (r+.z+ - r+.z) / r.z (Polak-Ribiere form, exact for a fixed linear preconditioner)
template <bool FLEX>
__global__ void __launch_bounds__(RB) k_cg_dir(CgArgs a)
{
    __shared__ double s_beta;
    const int rhs = blockIdx.y;
    const double *sc = a.sc + (size_t)rhs * S_COUNT;
    if (threadIdx.x < 32) {
        const double rz_new = fold(a.part, P_RZ, rhs, a.nrhs, a.nb);
        const double rz_mix = FLEX ? fold(a.part, P_AUX, rhs, a.nrhs, a.nb) : 0.0;
        if (threadIdx.x == 0) {
            const double rz_old = sc[S_RZ];
            s_beta = (sc[S_CONV] == 0.0 && rz_old > 0.0) ? (rz_new - rz_mix) / rz_old : 0.0;
        }
    }
    __syncthreads();
    const double beta = s_beta;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB) {
        const int64_t g = base + k;
        const double pv = a.z[g] + beta * a.p[g];
        a.p[g] = pv;
        a.p32[g] = (float)pv;
    }
}

// true residual f + L x (q64 = L x in FP64): partial ||.||^2 into P_AUX
__global__ void __launch_bounds__(RB) k_cg_true(CgArgs a)
{
    __shared__ double sh[RB / 32];
    const int rhs = blockIdx.y;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double ss = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB) {
        const double t = a.f[base + k] + a.q64[base + k];
        ss += t * t;
    }
    const double s = block_sum(ss, sh);
    if (threadIdx.x == 0) store_partial(a, P_AUX, rhs, s);
}

__global__ void k_cg_true_scalars(CgArgs a)
{
    const int rhs = blockIdx.x;
    if (threadIdx.x >= 32) return;
    const double ss = fold(a.part, P_AUX, rhs, a.nrhs, a.nb);
    if (threadIdx.x == 0) {
        double *sc = a.sc + (size_t)rhs * S_COUNT;
        sc[S_TRUE] = sc[S_FF] > 0.0 ? sqrt(ss / sc[S_FF]) : 0.0;
    }
}

// restart the right-hand sides whose true residual misses `goal`: r = f + L x and, unless
// FLEX (the network then recomputes z and k_cg_pz resets p), z = D^{-1} r, p = z
template <bool FLEX>
__global__ void __launch_bounds__(RB) k_cg_restart(CgArgs a, double goal)
{
    __shared__ double sh[RB / 32];
    const int rhs = blockIdx.y;
    const double *sc = a.sc + (size_t)rhs * S_COUNT;
    const bool redo = sc[S_TRUE] > goal;
    const int64_t base = seg_base(a, rhs), len = seg_len(a, rhs);
    double rz = 0.0, rr = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)RB + threadIdx.x; k < len; k += (int64_t)a.nb * RB) {
        const int64_t g = base + k;
        double rv = a.r[g];
        if (redo) {
            rv = a.f[g] + a.q64[g];
            a.r[g] = rv;
        }
        if (!FLEX) {
            double zv = a.z[g];
            if (redo) {
                zv = dinv_at(a, base, k) * rv;
                a.z[g] = zv;
                a.p[g] = zv;
                a.p32[g] = (float)zv;
            }
            rz += rv * zv;
        }
        rr += rv * rv;
    }
    double s;
    s = block_sum(rz, sh); if (threadIdx.x == 0 && !FLEX) store_partial(a, P_RZ, rhs, s);
    s = block_sum(rr, sh); if (threadIdx.x == 0) store_partial(a, P_RR, rhs, s);
    if (redo && blockIdx.x == 0 && threadIdx.x == 0)
        a.sc[(size_t)rhs * S_COUNT + S_CONV] = 0.0;
}

__global__ void k_invert(int64_t n, double *d, int have)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = have ? (d[i] > 0.0 ? 1.0 / d[i] : 1.0) : 1.0;
}

__global__ void k_zero(int64_t n, double *d)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) d[i] = 0.0;
}

}  // namespace

void nl_invert_launch(int64_t n, double *d, cudaStream_t st)
{
    k_invert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, d, 1);
}

nl_status nl_cg_state_release(nl_cg_state *c)
{
    if (c->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
    if (c->graph_exec_tail) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec_tail);
    if (c->ws) cudaFree(c->ws);
    if (c->ws32) cudaFree(c->ws32);
    if (c->red) cudaFree(c->red);
    if (c->host) cudaFreeHost(c->host);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->stream) cudaStreamDestroy(c->stream);
    memset(c, 0, sizeof(*c));
    return NL_OK;
}

nl_status nl_cg_release(nl_plan *p) { return nl_cg_state_release(&p->cg); }

struct EventPoll { cudaEvent_t ev; cudaError_t err; };

static int poll_event(void *ctx)
{
    EventPoll *e = (EventPoll *)ctx;
    e->err = cudaEventQuery(e->ev);
    if (e->err == cudaSuccess) return 1;
    return e->err == cudaErrorNotReady ? 0 : -1;
}

// bounded host wait on the chunk's event (nl_wait_poll with the library's wait limit): a chunk
// that does not finish in time returns NL_ETIMEOUT (its kernels keep running on the CG stream)
static nl_status wait_bounded(nl_cg_state *c)
{
    const double lim = nl_wait_limit_seconds();
    EventPoll ep{ c->ev, cudaSuccess };
    const nl_status s = nl_wait_poll(poll_event, &ep, lim);
    if (s == NL_ETIMEOUT)
        nl_set_error("nl_cg_solve: a chunk of iterations did not finish within %.3g s", lim);
    else if (s == NL_ECUDA)
        return nl_cuda_fail(ep.err, "CG chunk");
    return s;
}

static nl_status ensure_workspace(nl_cg_state *c, int64_t len, int64_t dlen, int nrhs)
{
    const size_t need64 = (size_t)4 * len + dlen;   // r z p q64 | dinv
    const size_t need32 = (size_t)2 * len;
    const size_t needr = (size_t)P_COUNT * nrhs * NB + (size_t)S_COUNT * nrhs;
    if (c->ws_elems >= need64 && c->ws32_elems >= need32 && c->red_elems >= needr &&
        c->host_elems >= (size_t)S_COUNT * nrhs && c->stream)
        return NL_OK;
    nl_cg_state_release(c);
    cudaError_t e;
    if ((e = cudaMalloc(&c->ws, need64 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->ws32, need32 * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c->red, needr * sizeof(double))) != cudaSuccess ||
        (e = cudaMallocHost(&c->host, (size_t)S_COUNT * nrhs * sizeof(double))) != cudaSuccess) {
        nl_cg_state_release(c);
        nl_set_error("nl_cg_solve: workspace allocation failed: %s", cudaGetErrorString(e));
        return NL_ENOMEM;
    }
    c->ws_elems = need64; c->ws32_elems = need32; c->red_elems = needr;
    c->host_elems = (size_t)S_COUNT * nrhs;
    NL_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    NL_CUDA_TRY(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
    return NL_OK;
}

static nl_status enqueue_chunk(nl_cg_op &op, const CgArgs &a, bool flex, int iters,
                               cudaStream_t st)
{
    const dim3 grid(a.nb, a.nrhs);
    for (int it = 0; it < iters; ++it) {
        nl_status s = op.apply(op.ctx, a.p32, a.q32, NL_F32, st);
        if (s != NL_OK) return s;
        k_cg_dot<<<grid, RB, 0, st>>>(a);
        if (flex) {
            k_cg_update<true><<<grid, RB, 0, st>>>(a);
            s = nl_net_apply_launch(op.net, op.net_plan, a.r, a.z, a.nrhs, st);
            if (s != NL_OK) return s;
            k_cg_rz<<<grid, RB, 0, st>>>(a);
            k_cg_dir<true><<<grid, RB, 0, st>>>(a);
        } else {
            k_cg_update<false><<<grid, RB, 0, st>>>(a);
            k_cg_dir<false><<<grid, RB, 0, st>>>(a);
        }
    }
    k_cg_check<<<a.nrhs, 32, 0, st>>>(a);
    NL_CUDA_TRY(cudaGetLastError());
    return NL_OK;
}

// The solver shared by nl_cg_solve, nl_cg_history and nl_batch_cg_solve.
nl_status nl_cg_run(nl_cg_op &op, const void *f, void *x, double rtol, int maxit, int precond,
                    double *hist, int cap, int *count, nl_cg_stats *stats, void *stream)
{
    const int nrhs = op.nrhs;
    if (!f || !x || nrhs < 1 || nrhs > 65535 || !(rtol > 0.0) || maxit < 0 ||
        precond < NL_PRECOND_NONE || precond > NL_PRECOND_LEARNED) {
        nl_set_error("nl_cg_solve: bad argument");
        return NL_EINVAL;
    }
    const bool flex = precond == NL_PRECOND_LEARNED;
    if (flex && (!op.net || !nl_net_valid(op.net))) {
        nl_set_error("nl_cg_solve: NL_PRECOND_LEARNED needs a network attached with "
                     "nl_plan_set_net on a symmetric 2-D scalar plan");
        return NL_EUNSUPPORTED;
    }
    nl_cg_state *c = op.state;
    const int64_t len = op.total;
    nl_status s = ensure_workspace(c, len, op.dinv_len, nrhs);
    if (s != NL_OK) return s;
    CgArgs a;
    a.per = op.per; a.seg_off = op.seg_off; a.seg_len = op.seg_len;
    a.dinv_global = op.seg_off ? 1 : 0;
    a.nrhs = nrhs;
    a.tol = 0.5 * rtol;
    a.f = (const double *)f; a.x = (double *)x;
    a.r = c->ws; a.z = a.r + len; a.p = a.z + len; a.q64 = a.p + len;
    double *dinv = a.q64 + len;          // [dinv_len], after the four vectors
    a.dinv = dinv;
    a.p32 = c->ws32; a.q32 = a.p32 + len;
    a.part = c->red; a.sc = c->red + (size_t)P_COUNT * nrhs * NB;
    // uniform segments: about CG_GRID_WAVES x NB blocks over all right-hand sides (each thread
    // then takes several elements); uneven segments keep NB each
    a.nb = op.seg_off ? NB
                      : std::max(16, std::min(NB, (CG_GRID_WAVES * NB + nrhs - 1) / nrhs));

    cudaStream_t caller = nl_stream(stream), st = c->stream;
    NL_CUDA_TRY(cudaEventRecord(c->ev, caller));
    NL_CUDA_TRY(cudaStreamWaitEvent(st, c->ev, 0));

    const unsigned g1 = (unsigned)((op.dinv_len + 255) / 256);
    k_zero<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(len, a.x);
    // the Jacobi factors depend on the operator only: formed once per workspace and mode
    const int dmode = precond != NL_PRECOND_NONE ? 2 : 1;
    if (c->dinv_at != dinv || c->dinv_mode != dmode) {
        c->dinv_at = nullptr;
        if (precond != NL_PRECOND_NONE) {
            s = op.diag(op.ctx, a.x, dinv, st);
            if (s != NL_OK) return s;
        }
        k_invert<<<g1, 256, 0, st>>>(op.dinv_len, dinv, precond != NL_PRECOND_NONE);
        NL_CUDA_TRY(cudaGetLastError());
        c->dinv_at = dinv;
        c->dinv_mode = dmode;
    }
    if (flex && (s = nl_net_reserve(op.net, op.net_plan, nrhs, st)) != NL_OK) return s;
    const dim3 grid(a.nb, nrhs);
    if (flex) {
        k_cg_init<true><<<grid, RB, 0, st>>>(a);
        k_cg_init_scalars<<<nrhs, 32, 0, st>>>(a);
        if ((s = nl_net_apply_launch(op.net, op.net_plan, a.r, a.z, nrhs, st)) != NL_OK) return s;
        k_cg_pz<<<grid, RB, 0, st>>>(a, -1, 0.0);
    } else {
        k_cg_init<false><<<grid, RB, 0, st>>>(a);
        k_cg_init_scalars<<<nrhs, 32, 0, st>>>(a);
    }
    NL_CUDA_TRY(cudaGetLastError());
    // one plain apply so that kernel attributes are set before capture
    s = op.apply(op.ctx, a.p32, a.q32, NL_F32, st);
    if (s != NL_OK) return s;

    // converged segments need no operator result inside the iterations (alpha = 0 freezes
    // them; a restart clears the flag before the next chunk reads it)
    if (op.set_skip) op.set_skip(op.ctx, a.sc + S_CONV, S_COUNT);
    // capture one chunk of iterations (the graph bakes in f, x, nrhs, the tolerance and the
    // preconditioner)
    if (c->graph_exec && (c->graph_nrhs != nrhs || c->graph_f != f || c->graph_x != x ||
                          c->graph_tol != rtol || c->graph_precond != precond ||
                          c->graph_net != (const void *)op.net ||
                          (op.net && c->graph_net_gen != nl_net_generation(op.net)))) {
        cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
        c->graph_exec = nullptr;
        if (c->graph_exec_tail) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec_tail);
        c->graph_exec_tail = nullptr;
    }
    auto capture = [&](int iters_in_graph, void **out) -> nl_status {
        cudaGraph_t g = nullptr;
        NL_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        nl_status cs = enqueue_chunk(op, a, flex, iters_in_graph, st);
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (cs != NL_OK) { if (g) cudaGraphDestroy(g); return cs; }
        if (ce != cudaSuccess) return nl_cuda_fail(ce, "cudaStreamEndCapture");
        cudaGraphExec_t ge = nullptr;
        ce = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return nl_cuda_fail(ce, "cudaGraphInstantiate");
        *out = ge;
        return NL_OK;
    };
    if (!c->graph_exec) {
        void *ge = nullptr, *gt = nullptr;
        if ((s = capture(CHUNK, &ge)) != NL_OK) return s;
        if ((s = capture(CHUNK_TAIL, &gt)) != NL_OK) {
            cudaGraphExecDestroy((cudaGraphExec_t)ge);
            return s;
        }
        c->graph_exec = ge;
        c->graph_exec_tail = gt;
        c->graph_nrhs = nrhs;
        c->graph_f = f;
        c->graph_x = x;
        c->graph_tol = rtol;
        c->graph_precond = precond;
        c->graph_net = op.net;
        c->graph_net_gen = op.net ? nl_net_generation(op.net) : 0;
    }

    double *h = c->host;
    int iters = 0, restarts = 0, snaps = 0;
    bool conv_all = false;
    const int64_t snap_len = op.per ? op.per : len;
    // shorter chunks once the recursive residual's decay predicts convergence within CHUNK
    // iterations (never with history snapshots, which keep the CHUNK cadence)
    bool tail = false;
    double prev_ratio = 0.0;
    int last_chunk = CHUNK;
    for (;;) {
        last_chunk = tail ? CHUNK_TAIL : CHUNK;
        NL_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)(tail ? c->graph_exec_tail : c->graph_exec),
                                    st));
        iters += last_chunk;
        if (hist && snaps < cap) {
            NL_CUDA_TRY(cudaMemcpyAsync(hist + (size_t)snaps * snap_len, a.x,
                                        snap_len * sizeof(double), cudaMemcpyDeviceToDevice, st));
            ++snaps;
        }
        NL_CUDA_TRY(cudaMemcpyAsync(h, a.sc, (size_t)S_COUNT * nrhs * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        NL_CUDA_TRY(cudaEventRecord(c->ev, st));
        if ((s = wait_bounded(c)) != NL_OK) return s;
        bool all = true;
        double ratio = 0.0;                  // largest r.r / f.f over the unconverged
        for (int r = 0; r < nrhs; ++r) {
            const double *hr = h + (size_t)r * S_COUNT;
            if (hr[S_CONV] == 0.0) {
                all = false;
                if (hr[S_FF] > 0.0) ratio = fmax(ratio, hr[S_RR] / hr[S_FF]);
            }
        }
        const bool out_of_budget = iters >= maxit;
        if (!all && !out_of_budget) {
            if (!hist && !tail && prev_ratio > 0.0 && ratio > 0.0 && ratio < prev_ratio) {
                const double per_it = std::log(ratio / prev_ratio) / last_chunk;   // < 0
                const double need = std::log(a.tol * a.tol / ratio) / per_it;
                if (need < CHUNK) tail = true;
            }
            prev_ratio = ratio;
            continue;
        }
        tail = false;
        prev_ratio = 0.0;
        // true FP64 residual f + L x
        s = op.apply(op.ctx, a.x, a.q64, NL_F64, st);
        if (s != NL_OK) return s;
        k_cg_true<<<grid, RB, 0, st>>>(a);
        k_cg_true_scalars<<<nrhs, 32, 0, st>>>(a);
        NL_CUDA_TRY(cudaMemcpyAsync(h, a.sc, (size_t)S_COUNT * nrhs * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        NL_CUDA_TRY(cudaEventRecord(c->ev, st));
        if ((s = wait_bounded(c)) != NL_OK) return s;
        double worst = 0.0;
        for (int r = 0; r < nrhs; ++r) worst = fmax(worst, h[r * S_COUNT + S_TRUE]);
        if (worst <= rtol) { conv_all = true; break; }
        if (out_of_budget || restarts >= 50) break;
        // defect correction: restart the right-hand sides that missed
        if (flex) {
            k_cg_restart<true><<<grid, RB, 0, st>>>(a, rtol);
            if ((s = nl_net_apply_launch(op.net, op.net_plan, a.r, a.z, nrhs, st)) != NL_OK) return s;
            k_cg_pz<<<grid, RB, 0, st>>>(a, 1, rtol);
        } else {
            k_cg_restart<false><<<grid, RB, 0, st>>>(a, rtol);
        }
        NL_CUDA_TRY(cudaGetLastError());
        ++restarts;
    }
    NL_CUDA_TRY(cudaStreamSynchronize(st));
    if (count) *count = snaps;
    if (stats) {
        int itmax = 0;
        double worst = 0.0;
        for (int r = 0; r < nrhs; ++r) {
            itmax = (int)fmax((double)itmax, h[r * S_COUNT + S_IT]);
            worst = fmax(worst, h[r * S_COUNT + S_TRUE]);
        }
        stats->iterations = itmax;
        stats->rel_residual = worst;
        stats->converged = conv_all ? 1 : 0;
    }
    if (!conv_all) {
        nl_set_error("nl_cg_solve: not converged to %g within %d iterations", rtol, maxit);
        return NL_ENOTCONV;
    }
    return NL_OK;
}

// ---- the plan's operator ----
struct PlanOpCtx { nl_plan *p; int nrhs; };

static nl_status plan_apply(void *ctx, const void *in, void *out, int dtype, cudaStream_t st)
{
    PlanOpCtx *c = (PlanOpCtx *)ctx;
    if (c->p->sym_fast) return nl_fast_sym_launch(c->p, in, out, c->nrhs, dtype, st);
    // the true residual: FP32-pair arithmetic where the plan has it (48-bit words, far below
    // the tolerances CG is asked for), FP64 otherwise
    if (dtype == NL_F64 && c->p->pair_rm)
        return nl_pairs_launch(c->p, (const double *)in, (double *)out, c->nrhs, st);
    return nl_direct_launch(c->p, in, out, c->nrhs, dtype, st);
}

// converged right-hand sides: the symmetric paired-column kernels skip their work items
static void plan_set_skip(void *ctx, const double *flags, int stride)
{
    nl_plan *p = ((PlanOpCtx *)ctx)->p;
    p->skip_flags = flags;
    p->skip_stride = stride;
}

static nl_status plan_diag(void *ctx, const double *zin, double *d, cudaStream_t st)
{
    nl_plan *p = ((PlanOpCtx *)ctx)->p;
    if (p->sym_fast) return nl_fast_sym_diag(p, d, st);
    return nl_diag_launch(p, zin, d, st);
}

static nl_status plan_cg(nl_plan *p, const void *f, void *x, int nrhs, double rtol, int maxit,
                         int precond, double *hist, int cap, int *count, nl_cg_stats *stats,
                         void *stream)
{
    if (!nl_plan_ok(p)) {
        nl_set_error("nl_cg_solve: invalid plan");
        return NL_EINVAL;
    }
    const bool pd = p->family == NL_PD_BOND;
    if (pd && p->d != 2) {
        nl_set_error("nl_cg_solve: the peridynamic operator of CG is the 2-D direct one");
        return NL_EUNSUPPORTED;
    }
    if (!(p->symmetric || p->sym_fast || (pd && p->const_horizon))) {
        nl_set_error("nl_cg_solve: the operator must be symmetric (symmetric NL_POWER or "
                     "NL_POLY plan, or NL_PD_BOND with a constant horizon)");
        return NL_EUNSUPPORTED;
    }
    if (precond == NL_PRECOND_LEARNED && (pd || p->d != 2 || p->sym_fast)) {
        nl_set_error("nl_cg_solve: NL_PRECOND_LEARNED needs a symmetric 2-D scalar plan");
        return NL_EUNSUPPORTED;
    }
    if (nrhs < 1 || nrhs > 65535) {
        nl_set_error("nl_cg_solve: bad argument");
        return NL_EINVAL;
    }
    PlanOpCtx ctx{ p, nrhs };
    nl_cg_op op;
    memset(&op, 0, sizeof(op));
    op.nrhs = nrhs;
    op.per = pd ? 2 * p->N : p->N;
    op.total = op.per * nrhs;
    op.dinv_len = op.per;
    op.apply = plan_apply;
    op.diag = plan_diag;
    op.ctx = &ctx;
    if (!pd && !p->sym_fast) op.set_skip = plan_set_skip;
    op.state = &p->cg;
    op.net = p->net;
    op.net_plan = p;
    const nl_status s = nl_cg_run(op, f, x, rtol, maxit, precond, hist, cap, count, stats,
                                   stream);
    plan_set_skip(&ctx, nullptr, 0);      // plain applies compute every right-hand side
    return s;
}

extern "C" nl_status nl_cg_solve(nl_plan *p, const void *f, void *x, int nrhs, double rtol,
                                 int maxit, int precond, nl_cg_stats *stats, void *stream)
{
    return plan_cg(p, f, x, nrhs, rtol, maxit, precond, nullptr, 0, nullptr, stats, stream);
}

extern "C" nl_status nl_cg_history(nl_plan *p, const void *f, void *x, double rtol, int maxit,
                                   int precond, double *history, int cap, int *count,
                                   nl_cg_stats *stats, void *stream)
{
    if (!history || cap < 1) {
        nl_set_error("nl_cg_history: need a history buffer with cap >= 1");
        return NL_EINVAL;
    }
    return plan_cg(p, f, x, 1, rtol, maxit, precond, history, cap, count, stats, stream);
}
