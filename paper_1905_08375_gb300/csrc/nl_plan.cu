// nl_plan.cu -- plan creation: validation, horizon data, offset tables,
// polynomial coefficients, exterior and self terms (host + plan-time kernels).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <new>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "nl_internal.cuh"

// ------------------------------------------------------------------------
// error reporting
// ------------------------------------------------------------------------
static thread_local char g_err[512];

void nl_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

nl_status nl_cuda_fail(cudaError_t e, const char *what)
{
    nl_set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return NL_ECUDA;
}

extern "C" const char *nl_last_error(void) { return g_err; }

// ------------------------------------------------------------------------
// failure handling on the host: injected host-allocation failures and the
// limit of the library's bounded host waits
// ------------------------------------------------------------------------
static std::atomic<long long> g_fail_after{ -1 };     // < 0: disarmed
static std::atomic<long long> g_wait_limit_ns{ 600LL * 1000000000LL };

bool nl_host_alloc_allowed()
{
    long long v = g_fail_after.load();
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v != 0;
    }
    return true;
}

extern "C" nl_status nl_debug_fail_host_alloc(int after)
{
    g_fail_after.store(after < 0 ? -1 : after);
    return NL_OK;
}

extern "C" nl_status nl_set_wait_limit(double seconds)
{
    if (!(seconds > 0.0) || seconds > 1.0e6) {
        nl_set_error("nl_set_wait_limit: need 0 < seconds <= 1e6 (got %g)", seconds);
        return NL_EINVAL;
    }
    g_wait_limit_ns.store((long long)(seconds * 1e9));
    return NL_OK;
}

double nl_wait_limit_seconds() { return (double)g_wait_limit_ns.load() * 1e-9; }

extern "C" nl_status nl_wait_poll(int (*poll)(void *ctx), void *ctx, double seconds)
{
    if (!poll) {
        nl_set_error("nl_wait_poll: null poll function");
        return NL_EINVAL;
    }
    if (!(seconds > 0.0)) seconds = nl_wait_limit_seconds();
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int r = poll(ctx);
        if (r > 0) return NL_OK;
        if (r < 0) {
            nl_set_error("nl_wait_poll: the polled condition reported an error (%d)", r);
            return NL_ECUDA;
        }
        const double dt =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > seconds) {
            nl_set_error("bounded wait gave up after %.3g s", seconds);
            return NL_ETIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// ------------------------------------------------------------------------
// constants of the kernel family
// ------------------------------------------------------------------------
static double unit_sphere_measure(int d)
{
    const double pi = 3.141592653589793238462643383279502884;
    return d == 1 ? 2.0 : (d == 2 ? 2.0 * pi : 4.0 * pi);
}

// Sec. 3 asks for the even polynomial p(s) = sum_m p_m s^{2m} whose value and
// first K derivatives at s = 1 match gamma(s) = s^{-alpha}.  With t = s^2 the
// map s -> t is smooth and invertible near s = 1, so matching K derivatives in
// s is the same as matching K derivatives in t: q(t) = p(sqrt t) must be the
// degree-K Taylor polynomial of t^{-alpha/2} at t = 1,
//   q(t) = sum_j binom(-alpha/2, j) (t - 1)^j,
// expanded here in powers of t.
static void hermite_poly(int K, double alpha, double *p)
{
    double taylor[9];
    double c = 1.0;
    for (int j = 0; j <= K; ++j) {
        taylor[j] = c;                          // binom(-alpha/2, j)
        c *= (-alpha / 2.0 - j) / (j + 1.0);
    }
    for (int m = 0; m <= K; ++m) p[m] = 0.0;
    // (t - 1)^j = sum_m binom(j, m) t^m (-1)^{j-m}
    for (int j = 0; j <= K; ++j) {
        double bjm = 1.0;
        for (int m = 0; m <= j; ++m) {
            if (m > 0) bjm = bjm * (j - m + 1) / m;
            p[m] += taylor[j] * bjm * (((j - m) & 1) ? -1.0 : 1.0);
        }
    }
}

// ------------------------------------------------------------------------
// plan-time kernels
// ------------------------------------------------------------------------
struct PlanArgs {
    int d, n, family, coef, symmetric, K;
    int64_t N;
    double alpha, sigma, h;
    double poly[8];
    int num_off;
    int Rmax;
};

__device__ __forceinline__ void node_coords(int64_t f, int d, int n, int c[3])
{
    c[0] = c[1] = c[2] = 0;
    for (int k = 0; k < d; ++k) { c[k] = (int)(f % n); f /= n; }
}

__device__ __forceinline__ double poly_eval_t(const double *pc, int K, double t)
{
    double r = pc[K];
    for (int m = K - 1; m >= 0; --m) r = r * t + pc[m];
    return r;
}

// Per-node horizon thresholds, computed in FP64 exactly as the ball test states:
// thr_i = largest integer < R2_i, thr4_i = largest integer < 4 R2_i.
__global__ void k_thresholds(PlanArgs a, const double *__restrict__ delta, int *thr, int *thr4)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    double rho = delta[i] * a.n;
    double R2 = rho * rho;
    thr[i] = (int)(ceil(R2) - 1.0);
    // clamp: with n <= 8192 every squared half-unit distance in Omega is below 2^30,
    // so a larger threshold selects the same cells
    if (thr4) thr4[i] = (int)fmin(ceil(4.0 * R2) - 1.0, 1073741824.0);
}

// Symmetric variant: a node's loop must reach every offset that lies in its own
// ball or in the ball of the node at that offset; bound it by the largest
// threshold in the (2 Rmax + 1)^d window.
__global__ void k_window_max(PlanArgs a, const int *__restrict__ thr, int *thr_win)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    int c[3];
    node_coords(i, a.d, a.n, c);
    int R = a.Rmax, m = thr[i];
    int z0 = a.d > 2 ? max(c[2] - R, 0) : 0, z1 = a.d > 2 ? min(c[2] + R, a.n - 1) : 0;
    int y0 = a.d > 1 ? max(c[1] - R, 0) : 0, y1 = a.d > 1 ? min(c[1] + R, a.n - 1) : 0;
    int x0 = max(c[0] - R, 0), x1 = min(c[0] + R, a.n - 1);
    for (int z = z0; z <= z1; ++z)
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                int64_t j = x + (int64_t)a.n * (y + (int64_t)a.n * z);
                m = max(m, thr[j]);
            }
    thr_win[i] = m;
}

// Per-node factors of the direct apply:
//   Lu_i = fin_i (sum_o wgt(o) (u_j - u_i) - u_i ext_i)
// POWER:  W_i = sigma h^{d-alpha} delta_i^{alpha-d-2},  g(o) = |o|^{-alpha}
// POLY:   W_i = sigma h^d delta_i^{-(d+2)},             g_i(o) = p(|o|^2 / R2_i)
// KAPPA:  W_i = sigma h^d delta_i^{-(d+2)},             g_i(o) = ra_i |o|^{-alpha} - p(|o|^2 / R2_i)
//         with ra_i = (delta_i / h)^alpha = R2_i^{alpha/2}, stored in the wh arrays
// one-sided: fin = A_i W_i, ext = b_ext E_i;  symmetric: fin = b_i, ext = b_i W_i E_i,
// with E_i = sum of g over the ball offsets whose node lies outside Omega.
__global__ void k_node_factors(PlanArgs a, const double *__restrict__ delta,
                               const double *__restrict__ coef, const int *__restrict__ thr,
                               const int *__restrict__ thr_loop, const int4 *__restrict__ off,
                               const double *__restrict__ gtab, int *cnt, float *b32,
                               double *b64, float *fin32, double *fin64, float *ext32,
                               double *ext64, float *wh32, double *wh64, float *ir32,
                               double *ir64)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const double di = delta[i];
    const double rho = di * a.n;
    const double R2 = rho * rho;
    const int t_i = thr[i];
    const int t_loop = thr_loop ? thr_loop[i] : t_i;
    // count of table entries with o2 <= t_loop (table sorted by o2)
    int lo = 0, hi = a.num_off;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (off[mid].w <= t_loop) lo = mid + 1; else hi = mid;
    }
    cnt[i] = lo;
    const double ai = coef ? coef[i] : 1.0;
    const double bi = (a.coef == NL_COEF_XY || a.coef == NL_COEF_MEAN) ? ai : 1.0;
    const double Ai = (a.coef == NL_COEF_X || a.coef == NL_COEF_XY) ? ai : 1.0;
    double W;
    if (a.family == NL_POWER)
        W = a.sigma * pow(a.h, a.d - a.alpha) * pow(di, a.alpha - a.d - 2.0);
    else
        W = a.sigma * pow(a.h, (double)a.d) * pow(di, -(a.d + 2.0));
    // exterior sum over this node's own ball
    int c[3];
    node_coords(i, a.d, a.n, c);
    int dist = c[0] < a.n - 1 - c[0] ? c[0] : a.n - 1 - c[0];
    for (int k = 1; k < a.d; ++k) dist = min(dist, min(c[k], a.n - 1 - c[k]));
    double E = 0.0;
    // the nearest exterior node is dist + 1 cells away along an axis
    if ((int64_t)(dist + 1) * (dist + 1) <= (int64_t)t_i) {
        for (int t = 0; t < a.num_off; ++t) {
            int4 o = off[t];
            if (o.w > t_i) break;
            bool out = (c[0] + o.x < 0) || (c[0] + o.x >= a.n);
            if (a.d > 1) out = out || (c[1] + o.y < 0) || (c[1] + o.y >= a.n);
            if (a.d > 2) out = out || (c[2] + o.z < 0) || (c[2] + o.z >= a.n);
            if (!out) continue;
            if (a.family == NL_POWER) E += gtab[t];
            else if (a.family == NL_KAPPA)
                E += pow(R2, 0.5 * a.alpha) * gtab[t] - poly_eval_t(a.poly, a.K, o.w / R2);
            else E += poly_eval_t(a.poly, a.K, o.w / R2);
        }
    }
    double fin, ext, wh = 0.0;
    if (a.symmetric) {
        fin = bi;
        ext = bi * W * E;
        wh = 0.5 * W;
    } else {
        fin = Ai * W;
        ext = bi * E;
        if (a.family == NL_KAPPA) wh = pow(R2, 0.5 * a.alpha);
    }
    b32[i] = (float)bi; b64[i] = bi;
    fin32[i] = (float)fin; fin64[i] = fin;
    ext32[i] = (float)ext; ext64[i] = ext;
    wh32[i] = (float)wh; wh64[i] = wh;
    ir32[i] = (float)(1.0 / R2); ir64[i] = 1.0 / R2;
}

// Peridynamic exterior sums: c_i * sum_{o in ball, node outside} o o^T / |o|^3.
__global__ void k_pd_exterior(PlanArgs a, const double *__restrict__ coef,
                              const int *__restrict__ thr, const int4 *__restrict__ off,
                              double *pdext)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    int c[3];
    node_coords(i, a.d, a.n, c);
    const int t_i = thr[i];
    double sxx = 0, sxy = 0, syy = 0;
    for (int t = 0; t < a.num_off; ++t) {
        int4 o = off[t];
        if (o.w > t_i) break;
        bool out = (c[0] + o.x < 0) || (c[0] + o.x >= a.n) || (c[1] + o.y < 0) ||
                   (c[1] + o.y >= a.n);
        if (!out) continue;
        double r = sqrt((double)o.w);
        double r3 = r * r * r;
        sxx += o.x * (double)o.x / r3;
        sxy += o.x * (double)o.y / r3;
        syy += o.y * (double)o.y / r3;
    }
    double ci = coef ? coef[i] : 1.0;
    pdext[3 * i + 0] = ci * sxx;
    pdext[3 * i + 1] = ci * sxy;
    pdext[3 * i + 2] = ci * syy;
}

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------
template <typename T>
static nl_status dev_alloc(nl_plan *p, T **ptr, size_t count)
{
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        nl_set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
        return NL_ENOMEM;
    }
    p->device_bytes += count * sizeof(T);
    return NL_OK;
}

#define NL_TRY(x)                          \
    do {                                   \
        nl_status _s = (x);                \
        if (_s != NL_OK) {                 \
            nl_plan_destroy(p);            \
            return _s;                     \
        }                                  \
    } while (0)

#define NL_CUDA_PLAN(call)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) {                             \
            nl_status _s = nl_cuda_fail(_e, #call);          \
            nl_plan_destroy(p);                              \
            return _s;                                       \
        }                                                    \
    } while (0)

static void free_tmp(double *a, double *b, int *c, int *d2)
{
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (c) cudaFree(c);
    if (d2) cudaFree(d2);
}

extern "C" nl_status nl_plan_create(nl_plan **out, const nl_grid *grid, const nl_horizon *hz,
                                    const nl_kernel *k, void *stream)
{
    if (!out || !grid || !hz || !k) {
        nl_set_error("nl_plan_create: null argument");
        return NL_EINVAL;
    }
    *out = nullptr;
    const int d = grid->dim, n = grid->n;
    if (d < 1 || d > 3 || n < 1) {
        nl_set_error("nl_plan_create: dim must be 1..3 and n >= 1 (got dim=%d n=%d)", d, n);
        return NL_EINVAL;
    }
    if (k->family < NL_POWER || k->family > NL_KAPPA) {
        nl_set_error("nl_plan_create: unknown kernel family %d", k->family);
        return NL_EINVAL;
    }
    if (k->coef < NL_COEF_NONE || k->coef > NL_COEF_MEAN) {
        nl_set_error("nl_plan_create: unknown coefficient mode %d", k->coef);
        return NL_EINVAL;
    }
    if (k->coef != NL_COEF_NONE && !k->a) {
        nl_set_error("nl_plan_create: coefficient mode %d needs the field a", k->coef);
        return NL_EINVAL;
    }
    if ((k->family == NL_POLY || k->family == NL_KAPPA || k->family == NL_PD_BOND) &&
        (k->K < 0 || k->K > 3)) {
        nl_set_error("nl_plan_create: K must be 0..3 (got %d)", k->K);
        return NL_EINVAL;
    }
    if (!(k->alpha >= 0.0) || !(k->alpha < d + 2.0) || !std::isfinite(k->scale)) {
        nl_set_error("nl_plan_create: need 0 <= alpha < d+2 and finite scale");
        return NL_EINVAL;
    }
    if (k->family == NL_PD_BOND) {
        // 2-D: the direct operator, the fast path and CG; 3-D: the fast path (nl_apply_fast,
        // K = 0, n = 2^L <= 256) only
        const bool pow2 = n >= 1 && (n & (n - 1)) == 0;
        if (d != 2 && !(d == 3 && pow2 && n <= 256 && k->K == 0)) {
            nl_set_error("nl_plan_create: the peridynamic operator is built for d = 2, and in "
                         "3-D for the fast path (K = 0, n = 2^L <= 256)");
            return NL_EUNSUPPORTED;
        }
        if (k->coef != NL_COEF_NONE && k->coef != NL_COEF_MEAN) {
            nl_set_error("nl_plan_create: peridynamic bonds take NL_COEF_NONE or NL_COEF_MEAN");
            return NL_EINVAL;
        }
    } else if (k->coef == NL_COEF_MEAN) {
        nl_set_error("nl_plan_create: NL_COEF_MEAN is for NL_PD_BOND");
        return NL_EINVAL;
    }
    if (hz->symmetric && k->family == NL_POLY) {
        // the symmetrised polynomial operator: the fast path with p = 1 (nl_apply_fast, CG)
        if (k->coef == NL_COEF_X || k->self_term != NL_SELF_DISCRETE) {
            nl_set_error("nl_plan_create: the symmetric NL_POLY variant needs "
                         "NL_COEF_NONE/XY and NL_SELF_DISCRETE");
            return NL_EUNSUPPORTED;
        }
    } else if (hz->symmetric && (k->family != NL_POWER || k->coef == NL_COEF_X)) {
        nl_set_error("nl_plan_create: the symmetric variant needs NL_POWER or NL_POLY with "
                     "NL_COEF_NONE/XY");
        return NL_EUNSUPPORTED;
    }
    int64_t N = 1;
    for (int q = 0; q < d; ++q) N *= n;
    if (N > ((int64_t)1 << 31) - 1) {
        nl_set_error("nl_plan_create: %lld nodes exceed the 2^31 limit", (long long)N);
        return NL_EUNSUPPORTED;
    }

    // ---- host-side horizon scan (validation of Eq. (2.3)) ----
    if (!nl_host_alloc_allowed()) {
        nl_set_error("nl_plan_create: host allocation of the horizon scan failed");
        return NL_ENOMEM;
    }
    std::vector<double> delta;
    try {
        delta.resize(N);
    } catch (const std::bad_alloc &) {
        nl_set_error("nl_plan_create: host allocation of the horizon scan failed");
        return NL_ENOMEM;
    }
    for (int64_t i = 0; i < N; ++i) delta[i] = hz->delta_field ? hz->delta_field[i] : hz->delta;
    int Rmax = 0;
    int64_t thr_max = 0;
    double rho_min = 1e300;
    for (int64_t i = 0; i < N; ++i) {
        double di = delta[i];
        if (!(di > 0.0) || !std::isfinite(di)) {
            nl_set_error("nl_plan_create: horizon must be > 0 and finite (node %lld: %g)",
                         (long long)i, di);
            return NL_EINVAL;
        }
        double rho = di * n;
        double R2 = rho * rho;
        if (R2 > 1.0e9) {
            nl_set_error("nl_plan_create: horizon of %g cells is beyond this build", rho);
            return NL_EUNSUPPORTED;
        }
        Rmax = std::max(Rmax, (int)std::ceil(rho));
        rho_min = std::min(rho_min, rho);
        thr_max = std::max(thr_max, (int64_t)(std::ceil(R2) - 1.0));
    }
    if (k->a) {
        for (int64_t i = 0; i < N; ++i)
            if (!(k->a[i] > 0.0) || !std::isfinite(k->a[i])) {
                nl_set_error("nl_plan_create: coefficient must be > 0 and finite (node %lld)",
                             (long long)i);
                return NL_EINVAL;
            }
    }

    nl_plan *p = nl_host_alloc_allowed() ? (nl_plan *)calloc(1, sizeof(nl_plan)) : nullptr;
    if (!p) {
        nl_set_error("nl_plan_create: host allocation failed");
        return NL_ENOMEM;
    }
    p->magic = NL_PLAN_MAGIC;
    p->version = NL_PLAN_VERSION;
    p->d = d; p->n = n; p->N = N;
    p->L = -1;
    for (int l = 0; l <= NL_MAX_LEVELS; ++l) if ((1 << l) == n) p->L = l;
    p->family = k->family; p->coef = k->coef; p->symmetric = hz->symmetric ? 1 : 0;
    if (p->symmetric && k->family == NL_POLY) {        // one-sided machinery + transpose half
        p->symmetric = 0;
        p->sym_fast = 1;
    }
    p->self_mode = k->self_term;
    p->K = (k->family == NL_POLY || k->family == NL_KAPPA || k->family == NL_PD_BOND) ? k->K : 0;
    if (k->fast_variant < NL_FAST_AUTO || k->fast_variant > NL_FAST_LEAFROWS) {
        nl_set_error("nl_plan_create: unknown fast variant %d", k->fast_variant);
        free(p);
        return NL_EINVAL;
    }
    p->fast_variant = k->fast_variant == NL_FAST_AUTO ? NL_FAST_LEAFROWS : k->fast_variant;
    p->alpha = k->alpha; p->scale = k->scale; p->h = 1.0 / n;
    if (k->family == NL_PD_BOND || !k->normalize)
        p->sigma = k->scale;
    else
        p->sigma = k->scale * 2.0 * d * (d + 2.0 - k->alpha) / unit_sphere_measure(d);
    if (k->family == NL_POLY || k->family == NL_KAPPA) hermite_poly(p->K, k->alpha, p->poly);
    if (k->family == NL_PD_BOND) hermite_poly(p->K, 3.0, p->poly);   // micromodulus ~ s^-3
    p->Rmax = Rmax;
    p->rho_min = rho_min;
    p->thr_max = (int)thr_max;
    p->const_horizon = 1;
    for (int64_t i = 1; i < N; ++i)
        if (delta[i] != delta[0]) { p->const_horizon = 0; break; }

    cudaStream_t st = nl_stream(stream);

    // ---- offset table: 0 < |o|^2 <= thr_max, sorted by |o|^2 then (dz, dy, dx) ----
    const int B = Rmax;
    std::vector<int4> offs;
    {
        const int bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
        for (int z = -bz; z <= bz; ++z)
            for (int y = -by; y <= by; ++y)
                for (int x = -B; x <= B; ++x) {
                    int64_t o2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                    if (o2 == 0 || o2 > thr_max) continue;
                    offs.push_back(make_int4(x, y, z, (int)o2));
                    if ((int64_t)offs.size() > NL_MAX_TABLE) {
                        nl_set_error("nl_plan_create: offset table beyond %d entries", NL_MAX_TABLE);
                        free(p);
                        return NL_EUNSUPPORTED;
                    }
                }
        std::stable_sort(offs.begin(), offs.end(), [](const int4 &a, const int4 &b) {
            if (a.w != b.w) return a.w < b.w;
            if (a.z != b.z) return a.z < b.z;
            if (a.y != b.y) return a.y < b.y;
            return a.x < b.x;
        });
    }
    p->num_off = (int)offs.size();

    // halo tile of the direct kernels
    int bx, by_, bz_;
    if (d == 1) { bx = DirectBlock<1>::X; by_ = 1; bz_ = 1; }
    else if (d == 2) { bx = DirectBlock<2>::X; by_ = DirectBlock<2>::Y; bz_ = 1; }
    else { bx = DirectBlock<3>::X; by_ = DirectBlock<3>::Y; bz_ = DirectBlock<3>::Z; }
    p->tile_sx = bx + 2 * B;
    p->tile_sy = d > 1 ? by_ + 2 * B : 1;
    p->tile_sz = d > 2 ? bz_ + 2 * B : 1;
    const size_t tile_elems = (size_t)p->tile_sx * p->tile_sy * p->tile_sz;
    size_t e32, e64;
    if (k->family == NL_PD_BOND) { e32 = 16; e64 = 32; }          // (ux, uy, c, -)
    else if (p->symmetric) { e32 = 16; e64 = 32; }                // (u, b, wh, thr)
    else { e32 = 8; e64 = 16; }                                   // (u, b)
    p->smem_bytes32 = tile_elems * e32;
    p->smem_bytes64 = tile_elems * e64;
    p->stage = (p->smem_bytes64 <= 200 * 1024) ? 1 : 0;
    if (d == 2 && k->family != NL_PD_BOND && (k->family != NL_KAPPA || k->K <= 1)) {
        // register-blocked kernel: (32 + 2R) x (32 + 2R + 8) tile + (2R+1)^2 weights
        const size_t t = (size_t)(32 + 2 * B) * (32 + 2 * B + 8);
        const size_t gw = (size_t)(2 * B + 1) * (2 * B + 1);
        p->rb_smem32 = t * e32 + gw * sizeof(float);
        p->rb_smem64 = t * e64 + gw * sizeof(double);
        p->rb2d = (p->rb_smem64 <= 200 * 1024) ? 1 : 0;
        // paired-column FP32 kernel: u and b planes of (64 + 2R) x (32 + 2R + 8) + weights
        p->x2_smem = (size_t)(64 + 2 * B) * (32 + 2 * B + 8) * 2 * sizeof(float) + gw * sizeof(float);
    }

    std::vector<OffEntry32> t32(offs.size());
    std::vector<OffEntry64> t64(offs.size());
    std::vector<double> g64(offs.size());
    std::vector<PdEntry32> q32;
    std::vector<PdEntry64> q64;
    for (size_t t = 0; t < offs.size(); ++t) {
        const int4 o = offs[t];
        int soff = o.x + p->tile_sx * (o.y + p->tile_sy * o.z);
        double g = (k->family == NL_POWER || k->family == NL_KAPPA)
                       ? std::pow((double)o.w, -k->alpha / 2.0) : 0.0;
        g64[t] = g;
        t32[t] = OffEntry32{ soff, o.w, (float)g, 0 };
        t64[t] = OffEntry64{ soff, o.w, g };
    }
    if (k->family == NL_PD_BOND && d == 2) {
        q32.resize(offs.size());
        q64.resize(offs.size());
        for (size_t t = 0; t < offs.size(); ++t) {
            const int4 o = offs[t];
            double r = std::sqrt((double)o.w), r3 = r * r * r;
            double gxx = o.x * (double)o.x / r3, gxy = o.x * (double)o.y / r3,
                   gyy = o.y * (double)o.y / r3;
            q32[t] = PdEntry32{ t32[t].soff, (float)gxx, (float)gxy, (float)gyy };
            q64[t] = PdEntry64{ t32[t].soff, 0, gxx, gxy, gyy };
        }
    }

    // ---- device uploads ----
    double *d_delta = nullptr, *d_a = nullptr, *d_g = nullptr;
    int *d_win = nullptr;
    auto fail_tmp = [&](nl_status s) {
        free_tmp(d_delta, d_a, nullptr, nullptr);
        if (d_g) cudaFree(d_g);
        nl_plan_destroy(p);
        return s;
    };
    if (cudaMalloc(&d_delta, N * sizeof(double)) != cudaSuccess) {
        nl_set_error("cudaMalloc failed for the horizon field");
        return fail_tmp(NL_ENOMEM);
    }
    if (k->a && cudaMalloc(&d_a, N * sizeof(double)) != cudaSuccess) {
        nl_set_error("cudaMalloc failed for the coefficient field");
        return fail_tmp(NL_ENOMEM);
    }
    if (cudaMalloc(&d_g, std::max<size_t>(1, g64.size()) * sizeof(double)) != cudaSuccess) {
        nl_set_error("cudaMalloc failed for the kernel table");
        return fail_tmp(NL_ENOMEM);
    }
    cudaError_t ce;
    ce = cudaMemcpyAsync(d_delta, delta.data(), N * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess && k->a)
        ce = cudaMemcpyAsync(d_a, k->a, N * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess && !g64.empty())
        ce = cudaMemcpyAsync(d_g, g64.data(), g64.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "plan upload"));

    nl_status s;
#define NL_TMP_TRY(x)                      \
    do {                                   \
        s = (x);                           \
        if (s != NL_OK) return fail_tmp(s); \
    } while (0)
    const size_t nt = std::max<size_t>(1, offs.size());
    NL_TMP_TRY(dev_alloc(p, &p->off, nt));
    NL_TMP_TRY(dev_alloc(p, &p->tab32, nt));
    NL_TMP_TRY(dev_alloc(p, &p->tab64, nt));
    NL_TMP_TRY(dev_alloc(p, &p->thr, N));
    NL_TMP_TRY(dev_alloc(p, &p->cnt, N));
    NL_TMP_TRY(dev_alloc(p, &p->b32, N));
    NL_TMP_TRY(dev_alloc(p, &p->b64, N));
    NL_TMP_TRY(dev_alloc(p, &p->fin32, N));
    NL_TMP_TRY(dev_alloc(p, &p->fin64, N));
    NL_TMP_TRY(dev_alloc(p, &p->ext32, N));
    NL_TMP_TRY(dev_alloc(p, &p->ext64, N));
    NL_TMP_TRY(dev_alloc(p, &p->wh32, N));
    NL_TMP_TRY(dev_alloc(p, &p->wh64, N));
    NL_TMP_TRY(dev_alloc(p, &p->ir32, N));
    NL_TMP_TRY(dev_alloc(p, &p->ir64, N));
    if (!offs.empty()) {
        ce = cudaMemcpyAsync(p->off, offs.data(), offs.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->tab32, t32.data(), t32.size() * sizeof(OffEntry32), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->tab64, t64.data(), t64.size() * sizeof(OffEntry64), cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "table upload"));
    }
    if (k->family == NL_PD_BOND && d == 2) {
        NL_TMP_TRY(dev_alloc(p, &p->pd32, nt));
        NL_TMP_TRY(dev_alloc(p, &p->pd64, nt));
        NL_TMP_TRY(dev_alloc(p, &p->pdext, 3 * N));
        if (!offs.empty()) {
            ce = cudaMemcpyAsync(p->pd32, q32.data(), q32.size() * sizeof(PdEntry32), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(p->pd64, q64.data(), q64.size() * sizeof(PdEntry64), cudaMemcpyHostToDevice, st);
            if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "pd table upload"));
        }
    }

    if (p->rb2d) {
        const int GW = 2 * B + 1;
        std::vector<float> g32(GW * GW);
        std::vector<double> gd(GW * GW);
        for (int oy = -B; oy <= B; ++oy)
            for (int ox = -B; ox <= B; ++ox) {
                const int o2 = ox * ox + oy * oy;
                const double g = (o2 == 0) ? 0.0 : std::pow((double)o2, -k->alpha / 2.0);
                gd[(ox + B) * GW + oy + B] = g;
                g32[(ox + B) * GW + oy + B] = (float)g;
            }
        NL_TMP_TRY(dev_alloc(p, &p->rb_g32, gd.size()));
        NL_TMP_TRY(dev_alloc(p, &p->rb_g64, gd.size()));
        ce = cudaMemcpyAsync(p->rb_g32, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->rb_g64, gd.data(), gd.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "weight table upload"));
    }

    if (k->family == NL_POWER && d == 3 && p->const_horizon && !p->symmetric && B <= 8) {
        // dense 3-D weight table |o|^{-alpha} for the slab kernel (0 at o = 0 and outside
        // the common ball), [oy][ox][oz]
        const int GW = 2 * B + 1;
        std::vector<float> g3((size_t)GW * GW * GW, 0.f);
        for (int oy = -B; oy <= B; ++oy)
            for (int ox = -B; ox <= B; ++ox)
                for (int oz = -B; oz <= B; ++oz) {
                    const int o2 = ox * ox + oy * oy + oz * oz;
                    if (o2 == 0 || o2 > p->thr_max) continue;
                    g3[((size_t)(oy + B) * GW + (ox + B)) * GW + (oz + B)] =
                        (float)std::pow((double)o2, -k->alpha / 2.0);
                }
        NL_TMP_TRY(dev_alloc(p, &p->g3d32, g3.size()));
        ce = cudaMemcpyAsync(p->g3d32, g3.data(), g3.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "3-D weight table upload"));
    }
    if (k->family == NL_PD_BOND && d == 2 && p->const_horizon && B <= 32) {
        // dense bond table for the paired-column FP32 kernel: (gxx, gxy, gyy) of every offset
        // of the (common) ball, zero outside it and at o = 0
        const int GW = 2 * B + 1;
        std::vector<float> gp((size_t)GW * GW * 3, 0.f);
        for (int ox = -B; ox <= B; ++ox)
            for (int oy = -B; oy <= B; ++oy) {
                const int o2 = ox * ox + oy * oy;
                if (o2 == 0 || o2 > p->thr_max) continue;
                const double r = std::sqrt((double)o2), r3 = r * r * r;
                float *e = &gp[((size_t)(ox + B) * GW + (oy + B)) * 3];
                e[0] = (float)(ox * (double)ox / r3);
                e[1] = (float)(ox * (double)oy / r3);
                e[2] = (float)(oy * (double)oy / r3);
            }
        NL_TMP_TRY(dev_alloc(p, &p->pd_dense32, gp.size()));
        ce = cudaMemcpyAsync(p->pd_dense32, gp.data(), gp.size() * sizeof(float), cudaMemcpyHostToDevice, st);
        if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "bond table upload"));
    }

    PlanArgs pa;
    pa.d = d; pa.n = n; pa.family = k->family; pa.coef = k->coef; pa.symmetric = p->symmetric;
    pa.K = p->K; pa.N = N; pa.alpha = k->alpha; pa.sigma = p->sigma; pa.h = p->h;
    for (int m = 0; m < 8; ++m) pa.poly[m] = p->poly[m];
    pa.num_off = p->num_off; pa.Rmax = Rmax;

    const int TB = 256;
    const unsigned GB = (unsigned)((N + TB - 1) / TB);
    const bool want_fast = (k->family == NL_POLY && p->L >= 0 && !p->symmetric);
    const bool want_fast_pd = (k->family == NL_PD_BOND && p->L >= 0 &&
                               ((d == 2 && n <= 8192) || (d == 3 && n <= 256 && k->K == 0)));
    if (want_fast || want_fast_pd) NL_TMP_TRY(dev_alloc(p, &p->thr4, N));
    k_thresholds<<<GB, TB, 0, st>>>(pa, d_delta, p->thr, p->thr4);
    if (p->symmetric) {
        NL_TMP_TRY(dev_alloc(p, &p->thr_reach, N));
        d_win = p->thr_reach;
        k_window_max<<<GB, TB, 0, st>>>(pa, p->thr, d_win);
    }
    k_node_factors<<<GB, TB, 0, st>>>(pa, d_delta, d_a, p->thr, d_win, p->off, d_g, p->cnt,
                                      p->b32, p->b64, p->fin32, p->fin64, p->ext32, p->ext64,
                                      p->wh32, p->wh64, p->ir32, p->ir64);
    if (k->family == NL_PD_BOND && d == 2)
        k_pd_exterior<<<GB, TB, 0, st>>>(pa, d_a, p->thr, p->off, p->pdext);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "plan kernels"));
    NL_TMP_TRY(nl_pairs_plan_init(p, offs.data(), g64.data(), (int)offs.size(), st));
    if (p->sym_fast && !want_fast) {
        nl_set_error("nl_plan_create: the symmetric NL_POLY variant needs n = 2^L");
        return fail_tmp(NL_EUNSUPPORTED);
    }
    if (want_fast) NL_TMP_TRY(nl_fast_plan_init(p, d_delta, d_a, st));
    if (p->sym_fast) {
        if (!p->pyr) {
            nl_set_error("nl_plan_create: no fast path for this grid (symmetric NL_POLY)");
            return fail_tmp(NL_EUNSUPPORTED);
        }
        NL_TMP_TRY(nl_fast_sym_plan_init(p, d_delta, d_a, st));
    }
    if (want_fast_pd) NL_TMP_TRY(nl_fast_pd_plan_init(p, d_delta, d_a, st));
    NL_TMP_TRY(nl_direct_plan_init(p, st));
    ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail_tmp(nl_cuda_fail(ce, "plan synchronise"));
    free_tmp(d_delta, d_a, nullptr, nullptr);
    cudaFree(d_g);
    *out = p;
    return NL_OK;
#undef NL_TMP_TRY
}

extern "C" nl_status nl_plan_destroy(nl_plan *p)
{
    if (!p) return NL_OK;
    if (!nl_plan_ok(p)) {
        nl_set_error("nl_plan_destroy: not a plan");
        return NL_EINVAL;
    }
    cudaDeviceSynchronize();
    void *ptrs[] = { p->thr, p->cnt, p->b32, p->b64, p->fin32, p->fin64, p->ext32, p->ext64,
                     p->wh32, p->wh64, p->ir32, p->ir64, p->off, p->tab32, p->tab64, p->pd32,
                     p->pd64, p->pdext, p->thr4, p->fastF, p->selfS, p->ir4, p->pyr, p->shift,
                     p->malpha, p->dinv64, p->rb_g32, p->rb_g64, p->thr_reach, p->fast_mx,
                     p->x2_order, p->x2_queue, p->pd_dense32, p->g3d32, p->leaf_multi,
                     p->aux_multi, p->fpd_F, p->fpd_M, p->fpd_P, p->fpd_aux, p->selfQ,
                     p->fastFh32, p->sym_c64, p->sym_c32, p->sym_T, p->sym_G64, p->sym_G32,
                     p->sym_diag, p->sym_D, p->sym_aux, p->sym_ir2, p->sym_P, p->kint_P, p->slot_base, p->slot_rec, p->slot_woff, p->slot_count,
                     p->fpd_ir2, p->pair_tab, p->pair_bc, p->x2r_order, p->x2r_queue,
                     p->x2r_c32, p->x2r_tp1, p->x2r_jmin };
    for (void *q : ptrs) if (q) cudaFree(q);
    for (int k = 0; k < 64; ++k)
        for (int j = 0; j < 3; ++j)
            if (p->prof_ev[k][j]) cudaEventDestroy(p->prof_ev[k][j]);
    nl_cg_release(p);
    p->magic = 0;
    free(p);
    return NL_OK;
}

extern "C" nl_status nl_get_plan_info(const nl_plan *p, nl_plan_info *info)
{
    if (!nl_plan_ok(p) || !info) {
        nl_set_error("nl_get_plan_info: bad plan or null info");
        return NL_EINVAL;
    }
    memset(info, 0, sizeof(*info));
    info->dim = p->d; info->n = p->n; info->levels = p->L;
    info->max_radius = p->Rmax; info->num_offsets = p->num_off;
    info->moments = p->M; info->sigma = p->sigma;
    for (int m = 0; m < 8; ++m) info->poly[m] = p->poly[m];
    info->device_bytes = p->device_bytes;
    info->step1_bytes = p->slots * (sizeof(unsigned) + 32 * sizeof(unsigned short));
    return NL_OK;
}
