// nl_internal.cuh -- plan layout and helpers shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "nl.h"

#define NL_PLAN_MAGIC 0x4e4c504cu  // "NLPL"
#define NL_PLAN_VERSION 1

// Largest supported ball radius (cells) and offset-table length.
#define NL_MAX_TABLE (1 << 20)
#define NL_MAX_LEVELS 20
#define NL_FAST_PARTS 1024

// Block shapes of the direct kernels: one output node per thread.
template <int D> struct DirectBlock;
template <> struct DirectBlock<1> { static constexpr int X = 128, Y = 1, Z = 1; };
template <> struct DirectBlock<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct DirectBlock<3> { static constexpr int X = 32, Y = 4, Z = 2; };

// One entry of the offset table, sorted by |o|^2.  soff is the offset inside
// the shared-memory halo tile of the direct kernels (strides fixed per plan).
struct __align__(16) OffEntry32 { int soff; int o2; float g; int pad; };
struct __align__(16) OffEntry64 { int soff; int o2; double g; };

// Peridynamic bond table: G = o o^T / |o|^3 (units of h), upper triangle.
struct __align__(16) PdEntry32 { int soff; float gxx, gxy, gyy; };
struct __align__(16) PdEntry64 { int soff; int pad; double gxx, gxy, gyy; };

// CG workspace and the captured graph of one chunk of iterations (owned by a plan or batch)
struct nl_cg_state {
    double *ws; size_t ws_elems;
    float *ws32; size_t ws32_elems;
    double *red; size_t red_elems;
    double *host; size_t host_elems;
    cudaStream_t stream;
    cudaEvent_t ev;
    void *graph_exec;               // cudaGraphExec_t: CHUNK iterations
    void *graph_exec_tail;          // the same for CHUNK_TAIL iterations (near convergence)
    int graph_nrhs;
    const void *graph_f, *graph_x;
    double graph_tol;
    int graph_precond;
    const void *graph_net;
    uint64_t graph_net_gen;
    const double *dinv_at;          // where the Jacobi factors were last formed (they are a
    int dinv_mode;                  // constant of the operator): 1 ones, 2 inverted diagonal
};

// The operator CG works with: nrhs segments (right-hand sides or batch instances) of the
// concatenated vectors; apply writes L in (FP32 or FP64), diag the FP64 diagonal of -L.
struct nl_cg_op {
    int nrhs;
    int64_t per;                    // uniform segment length (0 when seg_off/seg_len are used)
    int64_t total;                  // total length of the concatenated vectors
    const int64_t *seg_off, *seg_len;   // device arrays [nrhs], or nullptr for uniform
    int64_t dinv_len;               // per (uniform) or total
    nl_status (*apply)(void *ctx, const void *in, void *out, int dtype, cudaStream_t st);
    nl_status (*diag)(void *ctx, const double *zin, double *d, cudaStream_t st);
    void *ctx;
    nl_cg_state *state;
    // optional: segments whose flags[k * stride] is non-zero need no FP32 operator result
    // (called with the CG's convergence flags before the iterations, with null after)
    void (*set_skip)(void *ctx, const double *flags, int stride);
    nl_net *net;                    // flexible preconditioner (plan operators only)
    nl_plan *net_plan;
};
nl_status nl_cg_run(nl_cg_op &op, const void *f, void *x, double rtol, int maxit, int precond,
                    double *hist, int cap, int *count, nl_cg_stats *stats, void *stream);
nl_status nl_cg_state_release(nl_cg_state *c);

struct nl_plan {
    uint32_t magic;
    int version;
    // problem
    int d, n, L;            // L = log2 n or -1
    int64_t N;
    int family, coef, symmetric, self_mode, K, fast_variant;
    double alpha, scale, sigma, h;
    double poly[8];
    // horizon summary
    int Rmax;               // max ceil(delta_i n)
    double rho_min;         // min delta_i n
    int const_horizon;      // 1 if every node has the same horizon
    int thr_max;            // max over nodes of the largest integer |o|^2 inside the ball
    int num_off;            // table length (offsets with 0 < |o|^2 <= thr_sym_max)
    int stage;              // 1: direct kernels stage a halo tile in shared memory
    size_t smem_bytes32, smem_bytes64;
    int tile_sx, tile_sy, tile_sz;   // halo tile extents
    int rb2d;                       // 2-D register-blocked direct kernel usable
    size_t rb_smem32, rb_smem64, x2_smem;
    float *rb_g32; double *rb_g64;  // [2R+1][2R+1] kernel weights |o|^{-alpha} (0 at o = 0)
    float *pd_dense32;              // PD, 2-D, constant horizon: [2R+1][2R+1][3] bond tensors
    float *g3d32;                   // 3-D POWER, constant horizon: [2R+1]^3 weights (oy, ox, oz)
    int x3_var;                     // 3-D slab kernel variant (timed at plan creation)
    double *fpd_F, *fpd_M;          // fast-path PD: F_i and M_i (3 per node)
    double *fpd_ir2;                // fast-path PD, K >= 1: 1 / R_i^2 (R_i = delta_i n)
    long long *fpd_P;               // fast-path PD: ten leaf-row prefix arrays [10][N]
    void *fpd_aux;                  // fast-path PD: per-block bounds and the four scale exponents
    int fpd_bits;                   // fast-path PD: 2^bits >= n^2 (2 Rmax + 3)^2
    int *thr_reach;                 // symmetric variant: max threshold over the window
    int *x2_order, *x2_queue;       // paired-column FP32 kernel: tiles largest first, and the
    int x2_tiles, x2_blocks, x2_var;// work-queue counter + exit ticket; persistent grid size;
                                    // kernel variant (timed at plan creation)
    int *x2r_order, *x2r_queue;     // symmetric kernel for pairs of right-hand sides: 32-wide
    int x2r_tiles, x2r_blocks;      // tiles largest first, queue, tile count, grid size
    float *x2r_c32, *x2r_tp1;       // its tile planes c = (W/2) b and thr + 1 per node, and the
    int *x2r_jmin;                  // smallest threshold each tile stages
    const double *skip_flags;       // set by nl_cg_solve for its iterations only: right-hand
    int skip_stride;                // sides flagged converged need no FP32 operator result
    // per-node device arrays
    int *thr;               // largest integer < R2_i
    int *cnt;               // table entries with o2 <= thr_i (or the symmetric bound)
    float *b32;   double *b64;     // summed coefficient b_j (a_j or 1)
    float *fin32; double *fin64;   // final factor
    float *ext32; double *ext64;   // exterior coefficient
    float *wh32;  double *wh64;    // W_i / 2 (symmetric variant); (delta_i/h)^alpha (NL_KAPPA)
    float *ir32;  double *ir64;    // 1 / R2_i (polynomial kernels)
    // offset tables
    int4 *off;                      // (dx, dy, dz, o2)
    OffEntry32 *tab32; OffEntry64 *tab64;
    PdEntry32 *pd32; PdEntry64 *pd64;
    double *pdext;                  // [N][3] exterior G sums (xx, xy, yy) times c_i
    // fast path (Sec. 3)
    int M;                          // moments per panel
    int *thr4;                      // largest integer < 4 R2_i
    double *fastF;                  // sigma A_i delta_i^{-(d+2)}
    double *selfS;                  // self term S_i
    double *ir4;                    // 1 / (4 R2_i)
    double *pyr;                    // moment pyramid, levels 0..L, [panel][M]
    int64_t lvl_off[NL_MAX_LEVELS + 2];
    double *shift;                  // Step 2 re-centring table [2^d][M][M]
    int *malpha;                    // multi-indices [M][3]
    int pyr_rhs;                    // right-hand sides the pyramid buffer holds
    unsigned long long *fast_mx;    // FP32 integer route scratch: word 0 max |v| of the last
                                    // apply (fixed-point scale), word 1 a block ticket, then
                                    // NL_FAST_PARTS per-block maxima (floats, from byte 16)
    float fast_bmax;                // FP32 integer route: max |b| (bounds |u b| by max |u|)
    int r3_T4, r3_tm;               // 3-D constant horizon: the common threshold and the row
                                    // reach (= longest run) of the staged gather (tm 0: off)
    unsigned *slot_base;            // NL_FAST_PANELS, 1-D/2-D with n >= 32: the stored
    unsigned short *slot_rec;       // decomposition, warp-aligned slots (per-warp base
    int64_t *slot_woff;             // positions, per-node 16-bit records), per-warp slot
    int *slot_count;                // offsets and counts
    size_t slots;
    double *selfQ;                  // FP32 integer route: selfS / h^d and (float) fastF h^d
    float *fastFh32;
    long long *leaf_multi;          // leaf-row prefixes of several right-hand sides (grown on
    unsigned char *aux_multi;       // the first apply that needs them) and their scale words
    int leaf_multi_cap;
    // symmetrised fast path (K = 0): symmetric NL_POLY plans keep symmetric = 0 for the
    // one-sided machinery and set sym_fast
    int sym_fast;
    double *sym_c64; float *sym_c32;   // c_k = a_k delta_k^{-(d+2)}
    double *sym_T;                     // sum of c_k over the k whose leaf set reaches i
    double *sym_G64; float *sym_G32;   // sigma h^d a_i
    double *sym_diag;                  // Jacobi diagonal of -L
    double *sym_D;                     // difference arrays / row prefix sums (N x 8 bytes)
    unsigned char *sym_aux;            // scale word and per-block bounds of |c u|
    long long *kint_P;                 // one-sided K >= 1, FP32, d <= 2: [2K+1][N] leaf-row
    int kint_bits;                     // prefix sums of k^e q; 2^bits bounds a node's sums
    double *sym_ir2;                   // K >= 1: 1 / R_k^2 (R_k = delta_k n)
    long long *sym_P;                  // K >= 1: [2K+1][2][N] coefficient difference arrays
    int sym_limb;                      // K >= 1: bits of the low limb
    int sym_lgc;                       // K >= 1: ceil(log2(sources per target x weight bound))
    int prof_on, prof_count;        // per-phase timing of the fast apply
    cudaEvent_t prof_ev[64][3];
    int pair_rm;                    // NL_F64_PAIRS (2-D symmetric NL_POWER): tile halo, 0 = off
    float4 *pair_tab;               // offsets (tile offset, |o|^2, g hi, g lo)
    float4 *pair_bc;                // per node (b hi, b lo, c hi, c lo), c = W/2 b
    nl_cg_state cg;                 // CG workspace (allocated on the first solve)
    double *dinv64;                 // inverse Jacobi diagonal (computed on first use)
    double diag_mean;               // mean of the Jacobi diagonal (with dinv64)
    nl_net *net;                    // learned preconditioner (not owned)
    size_t device_bytes;
};

// ---- error reporting (thread-local message) ----
void nl_set_error(const char *fmt, ...);
nl_status nl_cuda_fail(cudaError_t e, const char *what);

// ---- host-side failure handling (nl_plan.cu) ----
// false once, when an injected host-allocation failure is due (nl_debug_fail_host_alloc)
bool nl_host_alloc_allowed();
// limit of the bounded host waits (nl_set_wait_limit; 600 s by default)
double nl_wait_limit_seconds();

#define NL_CUDA_TRY(call)                                                   \
    do {                                                                    \
        cudaError_t _e = (call);                                            \
        if (_e != cudaSuccess) return nl_cuda_fail(_e, #call);              \
    } while (0)

static inline bool nl_plan_ok(const nl_plan *p)
{
    return p && p->magic == NL_PLAN_MAGIC && p->version == NL_PLAN_VERSION;
}

static inline cudaStream_t nl_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ---- per-module launchers ----
nl_status nl_direct_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                           cudaStream_t st);
nl_status nl_pairs_plan_init(nl_plan *p, const int4 *offs, const double *g, int count,
                             cudaStream_t st);
nl_status nl_pairs_launch(const nl_plan *p, const double *u, double *Lu, int nrhs,
                          cudaStream_t st);
nl_status nl_pd_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                       cudaStream_t st);
nl_status nl_fast_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                         cudaStream_t st);
nl_status nl_direct_plan_init(nl_plan *p, cudaStream_t st);
nl_status nl_fast_pd_plan_init(nl_plan *p, const double *delta_dev, const double *c_dev,
                               cudaStream_t st);
nl_status nl_fast_pd_launch(nl_plan *p, const float *u, float *Lu, int nrhs, cudaStream_t st);
nl_status nl_fast_plan_init(nl_plan *p, const double *delta_dev, const double *a_dev,
                            cudaStream_t st);
nl_status nl_diag_launch(nl_plan *p, const double *zin, double *diag, cudaStream_t st);
nl_status nl_fast_sym_plan_init(nl_plan *p, const double *delta_dev, const double *a_dev,
                                cudaStream_t st);
nl_status nl_fast_sym_launch(nl_plan *p, const void *u, void *Lu, int nrhs, int dtype,
                             cudaStream_t st);
nl_status nl_fast_sym_diag(nl_plan *p, double *diag, cudaStream_t st);
nl_status nl_cg_release(nl_plan *p);
nl_status nl_batch_launch(int kind, int shape, int dtype, const void *inst_dev, int ninst,
                          int64_t total, int *counter, const void *u, void *Lu, int Rmax,
                          cudaStream_t st, const double *skip = nullptr, int skip_stride = 0);
nl_status nl_batch_fill_inst(nl_plan *const *plans, int count, const int64_t *offsets, int shape,
                             int dtype, int kind, void *host_out, int64_t *total_out);
size_t nl_batch_inst_bytes();
void nl_invert_launch(int64_t n, double *d, cudaStream_t st);
nl_status nl_net_apply_launch(nl_net *n, nl_plan *p, const double *r, double *z, int nrhs,
                              cudaStream_t st);
nl_status nl_net_reserve(nl_net *n, nl_plan *p, int nrhs, cudaStream_t st);
bool nl_net_valid(const nl_net *n);
// changes whenever a buffer address or a launch argument of the network's apply changes
uint64_t nl_net_generation(const nl_net *n);
