// nl_noalloc.cu -- nl_apply_fast_noalloc: the fast apply (p^0 = 1) for callers that may not
// allocate device memory.  No plan is created and nothing is allocated: every per-call work
// array (horizon thresholds, node factors, self terms and the Step 2 panel sums) lives in the
// file-scope device array below, whose size is fixed at build time.
//
// Some callers cannot call cudaMalloc: a host that has handed all device memory to its own
// pool allocator (a library cudaMalloc would fail or fragment that pool), or a caller on a
// latency-critical path that must not take the implicit device synchronisation cudaMalloc and
// cudaFree can cause.  They pass their inputs and outputs; the scratch is the array below.
//
// The array is part of this translation unit's device code, so every GPU on which the
// library's module is loaded holds NL_NOALLOC_SCRATCH_BYTES until the process exits.  All
// calls share it: two calls whose kernels overlap on the GPU (different streams, or different
// host threads, on one device) race on it and must be ordered by the caller.  Every value a
// call reads from the array is written earlier in the same call, so nothing needs clearing.
#include "nl_internal.cuh"

#define NL_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
// Largest horizon accepted, in units of the domain side.  A ball of radius 2 around any node
// covers Omega (whose diagonal is at most sqrt(3)); the bound keeps 4 (delta n)^2 below 2^30 for
// every accepted n (so the half-unit geometry stays in 32-bit integers) and the per-node
// self-term count (O((delta n)^{d-1}) row chords) small.
#define NL_NOALLOC_MAX_DELTA 2.0

static __device__ __align__(256) unsigned char g_nl_noalloc_scratch[NL_NOALLOC_SCRATCH_BYTES];

// The array's name in host code is only a stand-in for the symbol; the address a kernel may
// use comes from cudaGetSymbolAddress, looked up on every call with the caller's device
// current (it allocates nothing, and a module reloaded after cudaDeviceReset or a new primary
// context may place the array at a new address, so no address is cached).
static nl_status scratch_address(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_nl_noalloc_scratch);
    if (e != cudaSuccess || !p) return nl_cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    *out = (unsigned char *)p;
    return NL_OK;
}

namespace {

struct NaArgs {
    int d, n, L, self_mode;
    int64_t N;
    double delta_const, sigma, hd, sphere;
    const double *delta;          // device field or nullptr (constant horizon)
    int *thr4;                    // scratch
    double *fac, *selfS;          // scratch
    double *pyr;                  // scratch: levels 0..L-1 then the leaf level
    int64_t lvl_off[NL_MAX_LEVELS + 2];
};

__device__ __forceinline__ double na_delta(const NaArgs &a, int64_t i)
{
    return a.delta ? a.delta[i] : a.delta_const;
}

__device__ __forceinline__ int na_isqrt(int x)
{
    int r = (int)sqrtf((float)x);
    while (r > 0 && r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r;
}

// per node: threshold (largest integer below 4 R2, R2 = (delta n)^2 in FP64), factor
// sigma delta^{-(d+2)}, self term (continuous: |S^{d-1}| delta^d / d; discrete: h^d times
// the number of lattice cells, inside or outside Omega, that meet the open ball)
__global__ void k_na_nodes(NaArgs a)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const double di = na_delta(a, i);
    // field values outside (0, NL_NOALLOC_MAX_DELTA] (or NaN) are clamped for the geometry so
    // that the work stays bounded; such values are outside the documented range
    const double rho = fmin(fmax(di * a.n, 0.0), NL_NOALLOC_MAX_DELTA * a.n);
    const double R2 = rho * rho;
    const int T4 = (int)fmax(ceil(4.0 * R2) - 1.0, -1.0);
    a.thr4[i] = T4;
    a.fac[i] = a.sigma * pow(di, -(a.d + 2.0));
    if (a.self_mode == NL_SELF_PAPER) {
        a.selfS[i] = a.sphere * pow(di, (double)a.d) / a.d;
        return;
    }
    // lattice cells meeting the open ball: per row (fixed oy, oz) the cells with
    // (2|ox| - 1)^2 <= rest, i.e. |ox| <= (isqrt(rest) + 1) / 2, plus ox = 0
    const int B = (int)ceil(rho) + 1;
    const int bz = a.d > 2 ? B : 0, by = a.d > 1 ? B : 0;
    long long count = 0;
    for (int oz = -bz; oz <= bz; ++oz) {
        const long long gz = oz ? 2 * abs(oz) - 1 : 0;
        for (int oy = -by; oy <= by; ++oy) {
            const long long gy = oy ? 2 * abs(oy) - 1 : 0;
            const long long rest = (long long)T4 - gz * gz - gy * gy;
            if (rest < 0) continue;
            count += 2 * ((na_isqrt((int)rest) + 1) / 2) + 1;
        }
    }
    a.selfS[i] = a.hd * (double)count;
}

template <typename T>
__global__ void k_na_leaf(NaArgs a, const T *__restrict__ u)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < a.N) a.pyr[a.lvl_off[a.L] + i] = (double)u[i];
}

// Step 2 for p = 1: each parent panel holds the sum of its 2^d children
__global__ void k_na_level(NaArgs a, int l)
{
    const int np = 1 << l;
    int64_t P = np;
    if (a.d > 1) P *= np;
    if (a.d > 2) P *= np;
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= P) return;
    const int kx = (int)(f % np);
    const int ky = a.d > 1 ? (int)((f / np) % np) : 0;
    const int kz = a.d > 2 ? (int)(f / ((int64_t)np * np)) : 0;
    const int nc = 2 * np;
    const double *child = a.pyr + a.lvl_off[l + 1];
    double s = 0.0;
    for (int c = 0; c < (1 << a.d); ++c) {
        const int cx = 2 * kx + (c & 1);
        const int cy = a.d > 1 ? 2 * ky + ((c >> 1) & 1) : 0;
        const int cz = a.d > 2 ? 2 * kz + ((c >> 2) & 1) : 0;
        s += child[cx + (int64_t)nc * (cy + (int64_t)nc * cz)];
    }
    a.pyr[a.lvl_off[l] + f] = s;
}

// floor(a / 2^s) and ceil(a / 2^s) for signed a (arithmetic shift rounds toward -inf)
__device__ __forceinline__ int na_floor_shr(int a, int s) { return a >> s; }
__device__ __forceinline__ int na_ceil_shr(int a, int s) { return -((-a) >> s); }

__device__ __forceinline__ int na_far2(int k, int S, int X)
{
    const int p = abs(k * S - X), q = abs((k + 1) * S - X);
    const int m = p > q ? p : q;
    return m * m;
}
__device__ __forceinline__ int na_near2(int k, int S, int X)
{
    int g = 0;
    if (k * S > X) g = k * S - X;
    else if ((k + 1) * S < X) g = X - (k + 1) * S;
    return g * g;
}

// Step 1 + Step 3 for p = 1: per node, per level, per panel row, the panels whose parent is
// not fully inside the ball and that are fully inside it (or, at the leaf level, meet it)
template <int D, typename T>
__global__ void __launch_bounds__(256) k_na_gather(NaArgs a, const T *__restrict__ u,
                                                   T *__restrict__ Lu)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int n = a.n;
    const int ix = (int)(i % n);
    const int iy = D > 1 ? (int)((i / n) % n) : 0;
    const int iz = D > 2 ? (int)(i / ((int64_t)n * n)) : 0;
    const int X = 2 * ix + 1, Y = 2 * iy + 1, Z = 2 * iz + 1;
    const int T4 = a.thr4[i];
    const int r0 = na_isqrt(T4);
    double G = 0.0;
    for (int l = 0; l <= a.L; ++l) {
        const int np = 1 << l;
        const int sh = a.L - l + 1;        // panel size S = 2^sh half-units
        const int S = 1 << sh;
        const bool leaf = (l == a.L);
        const double *lev = a.pyr + a.lvl_off[l];
        int ylo = 0, yhi = 0, zlo = 0, zhi = 0;
        if (D > 1) {
            ylo = max(0, na_ceil_shr(Y - r0, sh) - (leaf ? 1 : 0));
            yhi = min(np - 1, na_floor_shr(Y + r0, sh) - (leaf ? 0 : 1));
        }
        if (D > 2) {
            zlo = max(0, na_ceil_shr(Z - r0, sh) - (leaf ? 1 : 0));
            zhi = min(np - 1, na_floor_shr(Z + r0, sh) - (leaf ? 0 : 1));
        }
        for (int kz = zlo; kz <= zhi; ++kz) {
            for (int ky = ylo; ky <= yhi; ++ky) {
                int e = 0;
                if (D > 1) e += leaf ? na_near2(ky, S, Y) : na_far2(ky, S, Y);
                if (D > 2) e += leaf ? na_near2(kz, S, Z) : na_far2(kz, S, Z);
                if (e > T4) continue;
                const int r = na_isqrt(T4 - e);
                int ka, kb;
                if (leaf) {
                    ka = max(0, na_ceil_shr(X - r, sh) - 1);
                    kb = min(np - 1, na_floor_shr(X + r, sh));
                } else {
                    ka = max(0, na_ceil_shr(X - r, sh));
                    kb = min(np - 1, na_floor_shr(X + r, sh) - 1);
                }
                if (ka > kb) continue;
                // panels of the parent row that are fully inside: excluded here
                int pa = 1, pb = 0;
                if (l > 0) {
                    int ep = 0;
                    if (D > 1) ep += na_far2(ky >> 1, 2 * S, Y);
                    if (D > 2) ep += na_far2(kz >> 1, 2 * S, Z);
                    if (ep <= T4) {
                        const int rp = na_isqrt(T4 - ep);
                        const int qa = max(0, na_ceil_shr(X - rp, sh + 1));
                        const int qb = min((np >> 1) - 1, na_floor_shr(X + rp, sh + 1) - 1);
                        if (qa <= qb) { pa = 2 * qa; pb = 2 * qb + 1; }
                    }
                }
                const double *row = lev + (int64_t)np * (ky + (int64_t)np * kz);
                for (int k = ka; k <= kb; ++k)
                    if (k < pa || k > pb) G += row[k];
            }
        }
    }
    Lu[i] = (T)(a.fac[i] * (a.hd * G - (double)u[i] * a.selfS[i]));
}

}  // namespace

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" nl_status nl_apply_fast_noalloc(int dim, int n, double delta, const double *delta_field,
                                           double alpha, double scale, int normalize,
                                           int self_term, const void *u, void *Lu, int nrhs,
                                           int dtype, void *stream)
{
    if (dim < 1 || dim > 3 || n < 1 || !u || !Lu || nrhs < 1 ||
        (dtype != NL_F32 && dtype != NL_F64) ||
        (self_term != NL_SELF_DISCRETE && self_term != NL_SELF_PAPER)) {
        nl_set_error("nl_apply_fast_noalloc: bad argument (dim 1..3, n >= 1, non-null u/Lu, "
                     "nrhs >= 1, dtype F32/F64, self term)");
        return NL_EINVAL;
    }
    if (!delta_field && !(delta > 0.0 && delta <= NL_NOALLOC_MAX_DELTA)) {
        nl_set_error("nl_apply_fast_noalloc: constant horizon must be in (0, %g] (got %g)",
                     NL_NOALLOC_MAX_DELTA, delta);
        return NL_EINVAL;
    }
    if (!(alpha >= 0.0 && alpha < dim + 2.0)) {
        nl_set_error("nl_apply_fast_noalloc: need 0 <= alpha < d + 2");
        return NL_EINVAL;
    }
    int L = -1;
    for (int l = 0; l <= 13; ++l) if ((1 << l) == n) L = l;
    if (L < 0) {
        nl_set_error("nl_apply_fast_noalloc: n must be a power of two <= 8192 (got %d)", n);
        return NL_EUNSUPPORTED;
    }
    NaArgs a;
    a.d = dim; a.n = n; a.L = L; a.self_mode = self_term;
    a.N = 1;
    for (int q = 0; q < dim; ++q) a.N *= n;
    // scratch layout: thresholds | factors | self terms | panel sums (levels 0..L)
    int64_t off = 0;
    for (int l = 0; l < L; ++l) {
        a.lvl_off[l] = off;
        int64_t P = 1;
        for (int q = 0; q < dim; ++q) P *= ((int64_t)1 << l);
        off += P;
    }
    a.lvl_off[L] = off;
    const size_t b_thr = align256((size_t)a.N * sizeof(int));
    const size_t b_fac = align256((size_t)a.N * sizeof(double));
    const size_t b_pyr = align256((size_t)(off + a.N) * sizeof(double));
    const size_t need = b_thr + 2 * b_fac + b_pyr;
    if (need > NL_NOALLOC_SCRATCH_BYTES) {
        nl_set_error("nl_apply_fast_noalloc: %lld nodes need %zu bytes of scratch, more than the "
                     "%zu-byte static array (at most 1-D n = 8192, 2-D n = 1024, 3-D n = 64)",
                     (long long)a.N, need, (size_t)NL_NOALLOC_SCRATCH_BYTES);
        return NL_EINVAL;
    }
    unsigned char *base = nullptr;
    nl_status s = scratch_address(&base);
    if (s != NL_OK) return s;
    a.thr4 = (int *)base;
    a.fac = (double *)(base + b_thr);
    a.selfS = (double *)(base + b_thr + b_fac);
    a.pyr = (double *)(base + b_thr + 2 * b_fac);
    const double pi = 3.141592653589793238462643383279502884;
    a.sphere = dim == 1 ? 2.0 : (dim == 2 ? 2.0 * pi : 4.0 * pi);
    a.sigma = normalize ? scale * 2.0 * dim * (dim + 2.0 - alpha) / a.sphere : scale;
    a.hd = 1.0;
    for (int q = 0; q < dim; ++q) a.hd /= n;
    a.delta = delta_field;
    a.delta_const = delta;

    cudaStream_t st = nl_stream(stream);
    const unsigned gb = (unsigned)((a.N + 255) / 256);
    k_na_nodes<<<gb, 256, 0, st>>>(a);
    NL_CUDA_TRY(cudaGetLastError());
    for (int r = 0; r < nrhs; ++r) {
        const size_t esz = dtype == NL_F32 ? sizeof(float) : sizeof(double);
        const void *ur = (const unsigned char *)u + (size_t)r * a.N * esz;
        void *lr = (unsigned char *)Lu + (size_t)r * a.N * esz;
        if (dtype == NL_F32) k_na_leaf<float><<<gb, 256, 0, st>>>(a, (const float *)ur);
        else k_na_leaf<double><<<gb, 256, 0, st>>>(a, (const double *)ur);
        for (int l = L - 1; l >= 0; --l) {
            int64_t P = 1;
            for (int q = 0; q < dim; ++q) P *= ((int64_t)1 << l);
            k_na_level<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(a, l);
        }
#define NL_NA_GATHER(D)                                                                         \
        do {                                                                                    \
            if (dtype == NL_F32)                                                                \
                k_na_gather<D, float><<<gb, 256, 0, st>>>(a, (const float *)ur, (float *)lr);   \
            else                                                                                \
                k_na_gather<D, double><<<gb, 256, 0, st>>>(a, (const double *)ur, (double *)lr);\
        } while (0)
        if (dim == 1) NL_NA_GATHER(1);
        else if (dim == 2) NL_NA_GATHER(2);
        else NL_NA_GATHER(3);
#undef NL_NA_GATHER
        NL_CUDA_TRY(cudaGetLastError());
    }
    return NL_OK;
}
