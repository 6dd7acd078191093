// fizzy_proj.cu -- host side of the C ABI declared in include/fizzy_proj.h:
// plan construction (grid metrics, eigenvalues, twiddles and z-factorisation
// tables built on the host in FP64), the kernel sequence of one projection,
// and the stats/error plumbing.
#include "fizzy_proj.h"
#include "kern_passes.cuh"
#include "kern_r16.cuh"
#include "kern_vc.cuh"
#include "kern_acdi.cuh"
#include "kern_probe.cuh"
#include "kern_poisson.cuh"
#include "kern_xy.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

using namespace fz;

namespace {

struct FFTHost {
    FFTDesc d64, d32;
    void *tw64 = nullptr, *tw32 = nullptr, *cs64 = nullptr, *cs32 = nullptr;
};

}  // namespace

// Pass kernels of a plan: the length-specialised instance where a direction
// is periodic with a length the library specialises (256, 512), else the
// generic one.  The results are the same bit for bit; only the index
// arithmetic differs.
typedef void (*XfwdK)(GridDev, FFTDesc, int, XArgs, int);
typedef void (*Ypass64K)(int, int, FFTDesc, int, double *, const int *, int, int);
typedef void (*Ypass32K)(int, int, FFTDesc, int, float *, const int *, int, int);
typedef void (*Xinv64K)(GridDev, FFTDesc, int, const double *, double *, const DevStats *, int);
typedef void (*Xinv32K)(GridDev, FFTDesc, int, const float *, double *, const DevStats *, int);
typedef void (*XYFwdK)(GridDev, XArgs);
typedef void (*XYInvK)(GridDev, const float *, double *, const DevStats *);
struct PassKernels {
    XfwdK xf64, xf32d, xf32l;
    XfwdK xl64;  // FP64 transform of a stored right-hand side (the preconditioner of fizzy_proj_solve_vc)
    Ypass64K yf64, yi64;
    Ypass32K yf32, yi32;
    Xinv64K xi64;
    Xinv32K xi32s, xi32a;
};

struct fizzy_proj_plan_s {
    fizzy_proj_desc desc;
    std::vector<double> zf;
    int mixed = 0, check = 0;
    double tol = 1e-10;
    double div_tol = 1e-10;
    int max_refine = 4;
    GridDev g;
    double sigma = 0.0;
    // device memory: one arena sized by plan_bytes, carved by dev_alloc
    // (later or larger requests get allocations of their own)
    std::vector<void *> allocs;
    unsigned char *arena = nullptr;
    size_t arena_size = 0, arena_off = 0;
    size_t bytes = 0;
    FFTHost fx, fy;
    int Ux = 0, Uy = 0;
    double *mtab64 = nullptr, *ibtab64 = nullptr, *cup64 = nullptr;
    float *mtab32 = nullptr, *ibtab32 = nullptr, *cup32 = nullptr;
    // periodic z: Sherman-Morrison weights and correction vector (k_ztables_cyc)
    double *wtab64 = nullptr, *qtab64 = nullptr;
    float *wtab32 = nullptr, *qtab32 = nullptr;
    // variable-coefficient solve (fizzy_proj_solve_vc), allocated on first use:
    // face beta x, y, z, r, z, d, A d, face rho x, y, z; partial sums; iteration state
    double *vc[10] = {};
    double *vc_part = nullptr;
    VcState *vc_state = nullptr;
    // ACDI step (fizzy_acdi_step), allocated on first use: psi, the unit
    // normal, sqrt((phi + delta)/(1 - phi + delta))
    double *acdi[5] = {};
    double *qx = nullptr, *qy = nullptr, *qz = nullptr;
    double *fhat64 = nullptr;
    float *fhat32 = nullptr;
    double *f = nullptr;
    DevStats *st = nullptr;
    double *usq_part = nullptr, *usq_sum = nullptr;
    int n_usq_part = 0;
    // end-to-end staging (solve_host, solve_host_async): two sets of the 7
    // device fields, two copy streams and their events, made on first use
    double *stage[2][7] = {};
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_done[2] = {}, ev_out[2] = {};
    bool set_used[2] = {false, false};
    int host_calls = 0;
    // launch shapes
    int Lx = 1, TXy = 2;
    int x_r16 = 0;  // mixed, nx of a register-resident length: register-resident FP32 x-passes
    int xthr32 = 256, ythr32 = 256;  // threads per CTA of the FP32 x- and y-pass kernels
    // mixed, nx = ny = 256 or 512, periodic or wall x/y: fused x-y cluster passes
    int xy_fused = 0;
    XYFwdK xyf_div = nullptr, xyf_load = nullptr;
    XYInvK xyi_store = nullptr, xyi_accum = nullptr;
    size_t xy_smem = 0;
    int xy_threads = 0;

    size_t smem_x64 = 0, smem_x32 = 0, smem_y64 = 0, smem_y32 = 0;
    int cap[24] = {0};  // resident-grid size of each pass kernel (CAP_*)
    PassKernels kern;   // the pass kernels this plan launches
    std::string err;
    // stream-ordered allocation (FIZZY_FLAG_ASYNC_ALLOC)
    int async_alloc = 0;
    cudaStream_t alloc_stream = nullptr;
    double *zt = nullptr;  // per-k tables (physics-dependent rows first)
    cudaError_t setup_err = cudaSuccess;  // first failed CUDA call while the plan is built
    // per-kernel timing
    int timing = 0;
    std::vector<cudaEvent_t> ev;        // 2 per recorded launch
    std::vector<int> ev_slot;           // kernel slot of each recorded launch
    int ev_used = 0;
    double t_ms[24] = {0};
    int t_cnt[24] = {0};
};

namespace {

enum {
    KS_FLUX, KS_XFWD, KS_YFWD, KS_THOMAS, KS_YINV, KS_XINV, KS_RESID, KS_XFWD_R, KS_YFWD_R,
    KS_THOMAS_R, KS_YINV_R, KS_XACC, KS_RCORR, KS_RESMAX, KS_CORRECT, KS_DIVMAX, KS_SUM, KS_N
};
const char *kSlotName[KS_N] = {"flux", "div_fwdx", "fwd_y", "thomas", "inv_y", "inv_x",
                               "resid", "fwd_x_refine", "fwd_y_refine", "thomas_refine",
                               "inv_y_refine", "inv_x_update", "resid_correct", "resid_check",
                               "correct", "div_check", "sum_partials"};
static_assert(KS_N <= 24, "timing slot arrays");
const int kMaxTimed = 8192;

const char *kErrStr[] = {"ok", "invalid argument", "unsupported size", "out of device memory",
                         "CUDA error", "not converged", "device wait timeout"};

bool radix23(int n) {
    if (n < 2) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

int set_err(fizzy_proj_plan_t p, int code, const std::string &msg) {
    if (p) p->err = msg;
    return code;
}

// The projection's staggered layout stores one face per cell and direction,
// so the near face of a direction is implicit: it takes periodic or wall x/y
// boundaries only.  The Dirichlet and mixed kinds are the Poisson solve's.
bool staggered_bcs(const fizzy_proj_desc &d) {
    return d.bc_x <= FIZZY_BC_NEUMANN && d.bc_y <= FIZZY_BC_NEUMANN;
}
const char *kNeedsStaggeredBcs =
    "this entry point takes periodic or wall x/y boundaries (Dirichlet kinds: fizzy_poisson_solve)";

// Keep the first failing CUDA call of plan construction (checked at its end).
void note(fizzy_proj_plan_t p, cudaError_t e) {
    if (e != cudaSuccess && p->setup_err == cudaSuccess) p->setup_err = e;
}

int cuda_err(fizzy_proj_plan_t p, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return set_err(p, FIZZY_ERR_CUDA, m);
}

template <typename T> T *dev_alloc(fizzy_proj_plan_t p, size_t count, int *status) {
    if (*status) return nullptr;
    void *ptr = nullptr;
    const size_t b = count * sizeof(T);
    const size_t ba = (b + 255) & ~(size_t)255;  // 256-byte aligned pieces
    if (p->arena && p->arena_off + ba <= p->arena_size) {
        ptr = p->arena + p->arena_off;
        p->arena_off += ba;
        p->bytes += b;
        return (T *)ptr;
    }
    cudaError_t e = p->async_alloc ? cudaMallocAsync(&ptr, b > 0 ? b : 16, p->alloc_stream)
                                   : cudaMalloc(&ptr, b > 0 ? b : 16);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *status = FIZZY_ERR_NOMEM;
        p->err = "cudaMalloc of " + std::to_string(b) + " bytes failed";
        return nullptr;
    }
    p->allocs.push_back(ptr);
    p->bytes += b;
    return (T *)ptr;
}

// Radix sequence of a Stockham plan: 4s first, then one 2, then 3s.
int make_radices(int n, int *rad) {
    int s = 0;
    while (n % 4 == 0) { rad[s++] = 4; n /= 4; }
    while (n % 2 == 0) { rad[s++] = 2; n /= 2; }
    while (n % 3 == 0) { rad[s++] = 3; n /= 3; }
    return s;
}

// Stage constants of an FFTDesc for length n (see FFTDesc).
void fill_stages(FFTDesc &d, int n) {
    d.n = n;
    d.nst = make_radices(n, d.rad);
    int ns = 1;
    for (int s = 0; s < d.nst; ++s) {
        d.m[s] = n / d.rad[s];
        d.ns[s] = ns;
        d.twq[s] = n / (ns * d.rad[s]);
        d.rm[s] = d.m[s] > 1 ? (unsigned)((1ull << 32) / (unsigned)d.m[s] + 1) : 0u;
        d.rns[s] = ns > 1 ? (unsigned)((1ull << 32) / (unsigned)ns + 1) : 0u;
        ns *= d.rad[s];
    }
    d.rn = (unsigned)((1ull << 32) / (unsigned)n + 1);
    d.rM = (unsigned)((1ull << 32) / (unsigned)(n / 2 + 1) + 1);
}

// Twiddle table entry t of length n in the form the Stockham stages use
// (kern_fft.cuh, tw_apply): w = exp(-2 pi i t / n) = c + i s is stored as
// (m, tau) with w = m (1 + i tau) when |c| >= |s| (R = 0) and
// w = i m (1 + i tau) otherwise (R = 1); R goes into the lowest mantissa bit
// of tau.  Computed in long double and rounded once.
void tw_entry(int n, int t, long double &m, long double &tau, int &R) {
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double a = 2.0L * pi * (long double)t / (long double)n;
    const long double c = cosl(a), sn = -sinl(a);
    if (fabsl(c) >= fabsl(sn)) {
        R = 0;
        m = c;
        tau = sn / c;
    } else {
        R = 1;
        m = sn;
        tau = -c / sn;
    }
}
double tw_tau64(long double tau, int R) {
    double v = (double)tau;
    uint64_t b;
    memcpy(&b, &v, 8);
    b = (b & ~1ull) | (uint64_t)R;
    memcpy(&v, &b, 8);
    return v;
}
float tw_tau32(long double tau, int R) {
    float v = (float)tau;
    uint32_t b;
    memcpy(&b, &v, 4);
    b = (b & ~1u) | (uint32_t)R;
    memcpy(&v, &b, 4);
    return v;
}

// Twiddles (n entries (m, tau)) and DCT post-twiddles (cos, sin)(pi m/(2n)),
// m = 0..n/2 (n/2+2 entries), into caller buffers; tw32/cs32 optional FP32 copies.
void fill_fft_tables(int n, double *tw, double *cs, float *tw32 = nullptr, float *cs32 = nullptr) {
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int t = 0; t < n; ++t) {
        long double m, tau;
        int R;
        tw_entry(n, t, m, tau, R);
        tw[2 * t] = (double)m;
        tw[2 * t + 1] = tw_tau64(tau, R);
        if (tw32) {
            tw32[2 * t] = (float)m;
            tw32[2 * t + 1] = tw_tau32(tau, R);
        }
    }
    for (int k = 0; k < n / 2 + 2; ++k) cs[2 * k] = cs[2 * k + 1] = 0.0;
    for (int k = 0; k <= n / 2; ++k) {
        const long double a = pi * (long double)k / (2.0L * (long double)n);
        cs[2 * k] = (double)cosl(a);
        cs[2 * k + 1] = (double)sinl(a);
    }
    if (cs32)
        for (int k = 0; k < 2 * (n / 2 + 2); ++k) cs32[k] = (float)cs[k];
}

// DCT-IV tables of a direction of length n (even, m = n/2): the m FFT
// twiddles of length m in the (m, tau) form, then the m pre-twiddles
// exp(-i pi (4t+1)/(4n)) as (cos, sin); cs: the m post-twiddles
// 2 exp(-i pi k/n).  Long double, rounded once.
void fill_dct4_tables(int n, double *tw, double *cs, float *tw32, float *cs32) {
    const long double pi = 3.141592653589793238462643383279502884L;
    const int m = n / 2;
    for (int t = 0; t < m; ++t) {
        long double mm, tau;
        int R;
        tw_entry(m, t, mm, tau, R);
        tw[2 * t] = (double)mm;
        tw[2 * t + 1] = tw_tau64(tau, R);
        tw32[2 * t] = (float)mm;
        tw32[2 * t + 1] = tw_tau32(tau, R);
        const long double a = -pi * (4.0L * t + 1.0L) / (4.0L * n);
        tw[2 * (m + t)] = (double)cosl(a);
        tw[2 * (m + t) + 1] = (double)sinl(a);
        tw32[2 * (m + t)] = (float)cosl(a);
        tw32[2 * (m + t) + 1] = (float)sinl(a);
    }
    for (int k = 0; k < n / 2 + 2; ++k) cs[2 * k] = cs[2 * k + 1] = 0.0;
    for (int k = 0; k < m; ++k) {
        const long double a = -pi * (long double)k / (long double)n;
        cs[2 * k] = (double)(2.0L * cosl(a));
        cs[2 * k + 1] = (double)(2.0L * sinl(a));
    }
    for (int k = 0; k < 2 * (n / 2 + 2); ++k) cs32[k] = (float)cs[k];
}

int build_fft(fizzy_proj_plan_t p, int n, int bc, FFTHost &F, int *status) {
    // the host tables of each length (and family) are computed once per process
    struct Tabs {
        std::vector<double> tw, cs;
        std::vector<float> tw32, cs32;
    };
    static std::mutex mu;
    static std::map<std::pair<int, int>, Tabs> cache;
    std::unique_lock<std::mutex> lock(mu);
    const bool dct4 = bc == FIZZY_BC_NEUMANN_DIRICHLET || bc == FIZZY_BC_DIRICHLET_NEUMANN;
    Tabs &T = cache[std::make_pair(n, dct4 ? 1 : 0)];
    if (T.tw.empty()) {
        T.tw.resize(2 * (size_t)n);
        T.cs.resize(2 * (size_t)(n / 2 + 2));
        T.tw32.resize(T.tw.size());
        T.cs32.resize(T.cs.size());
        if (dct4) fill_dct4_tables(n, T.tw.data(), T.cs.data(), T.tw32.data(), T.cs32.data());
        else fill_fft_tables(n, T.tw.data(), T.cs.data(), T.tw32.data(), T.cs32.data());
    }
    // ... and their device copies once per device: read-only, shared by every
    // plan of that length and family, kept for the life of the process
    struct DevTabs {
        void *tw64 = nullptr, *cs64 = nullptr, *tw32 = nullptr, *cs32 = nullptr;
    };
    static std::map<std::tuple<int, int, int>, DevTabs> dcache;
    int dev = 0;
    note(p, cudaGetDevice(&dev));
    DevTabs &D = dcache[std::make_tuple(dev, n, dct4 ? 1 : 0)];
    if (!D.tw64) {
        DevTabs t;
        const size_t b64 = T.tw.size() * sizeof(double), c64 = T.cs.size() * sizeof(double);
        const size_t b32 = T.tw32.size() * sizeof(float), c32 = T.cs32.size() * sizeof(float);
        cudaError_t e = cudaMalloc(&t.tw64, b64 + c64 + b32 + c32);
        if (e == cudaSuccess) {
            unsigned char *base = (unsigned char *)t.tw64;
            t.cs64 = base + b64;
            t.tw32 = base + b64 + c64;
            t.cs32 = base + b64 + c64 + b32;
            std::vector<unsigned char> h(b64 + c64 + b32 + c32);
            memcpy(h.data(), T.tw.data(), b64);
            memcpy(h.data() + b64, T.cs.data(), c64);
            memcpy(h.data() + b64 + c64, T.tw32.data(), b32);
            memcpy(h.data() + b64 + c64 + b32, T.cs32.data(), c32);
            e = cudaMemcpy(t.tw64, h.data(), h.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) cudaFree(t.tw64);
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *status = FIZZY_ERR_NOMEM;
            p->err = "twiddle tables: " + std::string(cudaGetErrorString(e));
            return *status;
        }
        D = t;
    }
    F.tw64 = D.tw64;
    F.cs64 = D.cs64;
    F.tw32 = D.tw32;
    F.cs32 = D.cs32;
    FFTDesc d;
    memset(&d, 0, sizeof(d));
    if (dct4) {  // stages of the half-length complex FFT; lines of length n
        fill_stages(d, n / 2);
        d.n = n;
        d.rn = (unsigned)((1ull << 32) / (unsigned)n + 1);
        d.rK = n / 2 > 1 ? (unsigned)((1ull << 32) / (unsigned)(n / 2) + 1) : 0u;
        d.kind = KIND_DCT4;
    } else {
        fill_stages(d, n);
        d.kind = (bc == FIZZY_BC_PERIODIC) ? KIND_PERIODIC : KIND_DCT;
    }
    d.flip = (bc == FIZZY_BC_DIRICHLET || bc == FIZZY_BC_DIRICHLET_NEUMANN) ? 1 : 0;
    F.d64 = d;
    F.d64.tw = F.tw64;
    F.d64.cs = F.cs64;
    F.d32 = d;
    F.d32.tw = F.tw32;
    F.d32.cs = F.cs32;
    return 0;
}

// Eigenvalue of the second difference at transform slot u:
//   periodic (half-complex index u)        -(4/h^2) sin^2(pi u / n)
//   Neumann both faces (DCT-II index u)    -(4/h^2) sin^2(pi u / (2n))
//   Dirichlet both faces (DST-II index n-1-u, see KIND_DCT's flip)
//                                          -(4/h^2) cos^2(pi u / (2n))
//   Neumann near, Dirichlet far (DCT-IV)   -(4/h^2) sin^2(pi (u + 1/2) / (2n))
//   Dirichlet near, Neumann far (DST-IV index n-1-u)
//                                          -(4/h^2) cos^2(pi (u + 1/2) / (2n))
double eig(int u, int n, double h, int bc) {
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double un = (long double)u, nn = (long double)n;
    long double s;
    switch (bc) {
        case FIZZY_BC_PERIODIC: s = sinl(pi * un / nn); break;
        case FIZZY_BC_NEUMANN: s = sinl(pi * un / (2.0L * nn)); break;
        case FIZZY_BC_DIRICHLET: s = cosl(pi * un / (2.0L * nn)); break;
        case FIZZY_BC_NEUMANN_DIRICHLET: s = sinl(pi * (un + 0.5L) / (2.0L * nn)); break;
        default: s = cosl(pi * (un + 0.5L) / (2.0L * nn)); break;
    }
    return (double)(-4.0L / ((long double)h * h) * s * s);
}

int validate(const fizzy_proj_desc *d) {
    if (!d) return FIZZY_ERR_INVALID;
    if (d->nx < 2 || d->ny < 2 || d->nz < 2) return FIZZY_ERR_INVALID;
    if (!(d->dx > 0) || !(d->dy > 0)) return FIZZY_ERR_INVALID;
    if (!d->zf && !(d->dz > 0)) return FIZZY_ERR_INVALID;
    if (d->bc_x < FIZZY_BC_PERIODIC || d->bc_x > FIZZY_BC_DIRICHLET_NEUMANN) return FIZZY_ERR_INVALID;
    if (d->bc_y < FIZZY_BC_PERIODIC || d->bc_y > FIZZY_BC_DIRICHLET_NEUMANN) return FIZZY_ERR_INVALID;
    if (d->periodic_z != 0 && d->periodic_z != 1) return FIZZY_ERR_INVALID;
    if (!(d->rho_l >= 1e-30 && d->rho_l <= 1e30) || !(d->rho_g >= 1e-30 && d->rho_g <= 1e30))
        return FIZZY_ERR_INVALID;
    if (!(d->dt > 0) || !std::isfinite(d->dt)) return FIZZY_ERR_INVALID;
    if (d->precision != FIZZY_PREC_FP64 && d->precision != FIZZY_PREC_MIXED) return FIZZY_ERR_INVALID;
    if (d->tol < 0 || d->max_refine < 0 || d->max_refine > 16) return FIZZY_ERR_INVALID;
    if (d->zf)
        for (int k = 0; k < d->nz; ++k)
            if (!(d->zf[k + 1] > d->zf[k])) return FIZZY_ERR_INVALID;
    if (!radix23(d->nx) || !radix23(d->ny)) return FIZZY_ERR_UNSUPPORTED;
    // the DCT-IV of a mixed direction runs as a complex FFT of half its length
    if (d->bc_x >= FIZZY_BC_NEUMANN_DIRICHLET && d->nx % 2) return FIZZY_ERR_UNSUPPORTED;
    if (d->bc_y >= FIZZY_BC_NEUMANN_DIRICHLET && d->ny % 2) return FIZZY_ERR_UNSUPPORTED;
    if (d->nx > FIZZY_MAX_N || d->ny > FIZZY_MAX_N) return FIZZY_ERR_UNSUPPORTED;
    if ((double)d->nx * d->ny * d->nz > 4.0e9) return FIZZY_ERR_UNSUPPORTED;
    // the (y, z) line index is split by a multiply-high division by ny, exact
    // below 2^32 / ny
    if ((double)d->ny * d->ny * d->nz >= 4294967296.0) return FIZZY_ERR_UNSUPPORTED;
    return FIZZY_OK;
}

// Physics-dependent scalars of GridDev (densities and dt; spacings dx, dy):
// shared by fizzy_proj_plan, fizzy_proj_set_physics and the allocation-free
// entry point.
void physics_consts(GridDev &g, double rho_l, double rho_g, double dt, double dx, double dy,
                    double sig) {
    const double rho0 = std::min(rho_l, rho_g), adrho = std::fabs(rho_l - rho_g);
    const bool var = adrho > 0.0;
    g.idt = 1.0 / dt;
    g.var_rho = var ? 1 : 0;
    // s'/r' lies in [1, 1 + |drho|/rho0]: centring the seed on half that range
    g.fsh = var ? (int)std::floor(0.5 * std::log2(1.0 + adrho / rho0)) : 0;
    g.fax = var ? rho0 * dx / dt : 0.0;
    g.frx = var ? 2.0 * rho0 * rho0 * dx / (dt * adrho) : 0.0;
    g.fay = var ? rho0 * dy / dt : 0.0;
    g.fry = var ? 2.0 * rho0 * rho0 * dy / (dt * adrho) : 0.0;
    g.dvx = rho0 / (dt * dx);
    g.dvy = rho0 / (dt * dy);
    g.dvx_s = sig * rho0 / (dt * dx);
    g.dvy_s = sig * rho0 / (dt * dy);
    g.dt = dt;
    g.cgx = dt / (rho0 * dx);
    g.cgy = dt / (rho0 * dy);
    g.div_scale = dt / rho0 * dx;
}

// The physics rows of the per-k tables at plane k (the first kZPhys rows of
// the table block): a' and r' of the z face above k, rho0/(dt dzf_k),
// sigma rho0/(dt dzf_k), dt/(rho0 dzc_(k+1/2)).  dzc is the centre distance
// to plane k+1 (unused on the top plane).
constexpr int kZPhys = 5;
void physics_zrow(double rho_l, double rho_g, double dt, double sig, double dzf, double dzc,
                  bool top, double *row, size_t stride) {
    const double rho0 = std::min(rho_l, rho_g), adrho = std::fabs(rho_l - rho_g);
    const bool face = !top && adrho > 0.0;
    const double idzc = top ? 0.0 : 1.0 / dzc;
    row[0 * stride] = face ? rho0 * dzc / dt : 0.0;
    row[1 * stride] = face ? 2.0 * rho0 * rho0 * dzc / (dt * adrho) : 0.0;
    row[2 * stride] = rho0 / (dt * dzf);
    row[3 * stride] = sig * rho0 / (dt * dzf);
    row[4 * stride] = dt / rho0 * idzc;
}

// Grid of a stand-alone pass launch: the CTAs of the kernel the GPU holds
// resident (occupancy x SM count); the kernel strides over its tiles.
enum { CAP_XF64, CAP_XF32D, CAP_XF32L, CAP_Y64F, CAP_Y64I, CAP_Y32F, CAP_Y32I, CAP_XI64, CAP_XI32S,
       CAP_XI32A, CAP_TH64, CAP_TH32, CAP_TH64C, CAP_TH32C, CAP_RM, CAP_RC, CAP_CIF, CAP_N };
// Cached per (device, kernel, block size, shared memory): plans are built per
// request in the serving runtime, and the occupancy queries would dominate.
template <typename K> int resident_grid(K kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, (const void *)kernel, threads, smem);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int sms = 0, nb = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        nb = 1;
    }
    const int g = std::max(1, nb) * std::max(1, sms);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = g;
    return g;
}
template <typename T> size_t pass_smem(int n, int L) {
    return sizeof(typename C2<T>::t) * ((size_t)n + (n / 2 + 2) + 2 * (size_t)L * (n + 1));
}

// The specialised length of a direction (0: generic).
int fixed_len(int n, int bc) { return (bc == FIZZY_BC_PERIODIC && (n == 256 || n == 512)) ? n : 0; }

template <int NX, int NY> PassKernels kernels_for() {
    PassKernels k;
    k.xf64 = k_xfwd<double, XF_F64_DIVQ, NX>;
    k.xf32d = k_xfwd<float, XF_MIX_DIVQ, NX>;
    k.xf32l = k_xfwd<float, XF_MIX_LOAD, NX>;
    k.xl64 = k_xfwd<double, XF_MIX_LOAD, NX>;
    k.yf64 = k_ypass<double, false, NY>;
    k.yi64 = k_ypass<double, true, NY>;
    k.yf32 = k_ypass<float, false, NY>;
    k.yi32 = k_ypass<float, true, NY>;
    k.xi64 = k_xinv<double, XI_STORE, NX>;
    k.xi32s = k_xinv<float, XI_STORE, NX>;
    k.xi32a = k_xinv<float, XI_ACCUM, NX>;
    return k;
}
template <int NX> PassKernels kernels_for_y(int fy) {
    return fy == 256 ? kernels_for<NX, 256>() : fy == 512 ? kernels_for<NX, 512>() : kernels_for<NX, 0>();
}
PassKernels pick_kernels(int fx, int fy) {
    return fx == 256 ? kernels_for_y<256>(fy) : fx == 512 ? kernels_for_y<512>(fy) : kernels_for_y<0>(fy);
}

// The length of a direction that has register-resident FP32 passes
// (periodic or Neumann; 0: none).
int r_len(int n) { return r_supported(n) ? n : 0; }

// Mixed plans: the register-resident FP32 passes (static shared memory, no
// opt-in) replace the Stockham ones along a direction of a supported
// length.
template <int N, int KIND> void r_kernels_x(PassKernels &k) {
    k.xf32d = k_xfwd_r_divq<N, KIND>;
    k.xf32l = k_xfwd_r_load<N, KIND>;
    k.xi32s = k_xinv_r<XI_STORE, N, KIND>;
    k.xi32a = k_xinv_r<XI_ACCUM, N, KIND>;
}
template <int N, int KIND> void r_kernels_y(PassKernels &k) {
    k.yf32 = k_ypass_r<false, N, KIND>;
    k.yi32 = k_ypass_r<true, N, KIND>;
}
template <int N> void r_kernels_xn(PassKernels &k, bool dct) {
    dct ? r_kernels_x<N, KIND_DCT>(k) : r_kernels_x<N, KIND_PERIODIC>(k);
}
template <int N> void r_kernels_yn(PassKernels &k, bool dct) {
    dct ? r_kernels_y<N, KIND_DCT>(k) : r_kernels_y<N, KIND_PERIODIC>(k);
}
void pick_r_kernels(PassKernels &k, int nx, int bcx, int ny, int bcy) {
    const bool dx = bcx == FIZZY_BC_NEUMANN, dy = bcy == FIZZY_BC_NEUMANN;
    switch (nx) {
    case 32: r_kernels_xn<32>(k, dx); break;
    case 48: r_kernels_xn<48>(k, dx); break;
    case 64: r_kernels_xn<64>(k, dx); break;
    case 96: r_kernels_xn<96>(k, dx); break;
    case 128: r_kernels_xn<128>(k, dx); break;
    case 192: r_kernels_xn<192>(k, dx); break;
    case 256: r_kernels_xn<256>(k, dx); break;
    case 384: r_kernels_xn<384>(k, dx); break;
    case 512: r_kernels_xn<512>(k, dx); break;
    default: break;
    }
    switch (ny) {
    case 32: r_kernels_yn<32>(k, dy); break;
    case 48: r_kernels_yn<48>(k, dy); break;
    case 64: r_kernels_yn<64>(k, dy); break;
    case 96: r_kernels_yn<96>(k, dy); break;
    case 128: r_kernels_yn<128>(k, dy); break;
    case 192: r_kernels_yn<192>(k, dy); break;
    case 256: r_kernels_yn<256>(k, dy); break;
    case 384: r_kernels_yn<384>(k, dy); break;
    case 512: r_kernels_yn<512>(k, dy); break;
    default: break;
    }
}

// The fused x-y cluster kernels of a length and transform kinds.
template <int N, int KX, int KY> void xy_kernels(XYFwdK *fd, XYFwdK *fl, XYInvK *is, XYInvK *ia) {
    *fd = k_xy_fwd<N, KX, KY, XY_DIVQ>;
    *fl = k_xy_fwd<N, KX, KY, XY_LOAD>;
    *is = k_xy_inv<N, KX, KY, XI_STORE>;
    *ia = k_xy_inv<N, KX, KY, XI_ACCUM>;
}
template <int N> void xy_kernels_n(int kx, int ky, XYFwdK *fd, XYFwdK *fl, XYInvK *is, XYInvK *ia) {
    if (kx == KIND_PERIODIC && ky == KIND_PERIODIC) xy_kernels<N, KIND_PERIODIC, KIND_PERIODIC>(fd, fl, is, ia);
    else if (kx == KIND_PERIODIC) xy_kernels<N, KIND_PERIODIC, KIND_DCT>(fd, fl, is, ia);
    else if (ky == KIND_PERIODIC) xy_kernels<N, KIND_DCT, KIND_PERIODIC>(fd, fl, is, ia);
    else xy_kernels<N, KIND_DCT, KIND_DCT>(fd, fl, is, ia);
}
// Set up the fused passes of a plan when its shape allows them and the
// device runs the clusters: opt the kernels into their shared memory (once
// per device) and check that a cluster fits.  Returns 1 if enabled.
int setup_xy(fizzy_proj_plan_t p, int n, int kx, int ky) {
    XYFwdK fd, fl;
    XYInvK is, ia;
    size_t smem;
    int threads;
    if (n == 512) {
        xy_kernels_n<512>(kx, ky, &fd, &fl, &is, &ia);
        smem = xy_smem_bytes<512>();
        threads = XYShape<512>::THREADS;
    } else {
        xy_kernels_n<256>(kx, ky, &fd, &fl, &is, &ia);
        smem = xy_smem_bytes<256>();
        threads = XYShape<256>::THREADS;
    }
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> ok_cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(dev, (const void *)fd);
    auto it = ok_cache.find(key);
    int ok;
    if (it != ok_cache.end()) {
        ok = it->second;
    } else {
        ok = 1;
        for (const void *f : {(const void *)fd, (const void *)fl, (const void *)is, (const void *)ia})
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                ok = 0;
        if (ok) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(XY_CL);
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = smem;
            int nclusters = 0;
            for (const void *f : {(const void *)fd, (const void *)fl, (const void *)is, (const void *)ia}) {
                if (cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg) != cudaSuccess || nclusters < 1) ok = 0;
            }
        }
        (void)cudaGetLastError();
        ok_cache[key] = ok;
    }
    if (!ok) return 0;
    p->xyf_div = fd;
    p->xyf_load = fl;
    p->xyi_store = is;
    p->xyi_accum = ia;
    p->xy_smem = smem;
    p->xy_threads = threads;
    return 1;
}

// Opt every pass kernel instance into large dynamic shared memory.
void opt_in_smem(fizzy_proj_plan_t p, int bytes) {
    for (int fx : {0, 256, 512})
        for (int fy : {0, 256, 512}) {
            const PassKernels k = pick_kernels(fx, fy);
            const void *fns[] = {(const void *)k.xf64, (const void *)k.xf32d, (const void *)k.xf32l,
                                 (const void *)k.xl64,
                                 (const void *)k.yf64, (const void *)k.yi64, (const void *)k.yf32,
                                 (const void *)k.yi32, (const void *)k.xi64, (const void *)k.xi32s,
                                 (const void *)k.xi32a};
            for (const void *f : fns)
                note(p, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        }
}

// sx32r: dynamic shared memory of the FP32 x-passes (0 for the
// register-resident ones)
void pass_caps(int *cap, const PassKernels &k, size_t sx64, size_t sx32, size_t sx32r, size_t sy64,
               size_t sy32, int tx32, int ty32) {
    cap[CAP_XF64] = resident_grid(k.xf64, 256, sx64);
    cap[CAP_XF32D] = resident_grid(k.xf32d, tx32, sx32r);
    cap[CAP_XF32L] = resident_grid(k.xf32l, tx32, sx32r);
    cap[CAP_Y64F] = resident_grid(k.yf64, 256, sy64);
    cap[CAP_Y64I] = resident_grid(k.yi64, 256, sy64);
    cap[CAP_Y32F] = resident_grid(k.yf32, ty32, sy32);
    cap[CAP_Y32I] = resident_grid(k.yi32, ty32, sy32);
    cap[CAP_XI64] = resident_grid(k.xi64, 256, sx64);
    cap[CAP_XI32S] = resident_grid(k.xi32s, tx32, sx32r);
    cap[CAP_XI32A] = resident_grid(k.xi32a, tx32, sx32r);
    cap[CAP_TH64] = resident_grid(k_thomas<double>, THOMAS_BLOCK, thomas_smem<double>());
    cap[CAP_TH32] = resident_grid(k_thomas<float>, THOMAS_BLOCK, thomas_smem<float>());
    cap[CAP_TH64C] = resident_grid(k_thomas_cyc<double>, THOMAS_BLOCK, thomas_cyc_smem<double>());
    cap[CAP_TH32C] = resident_grid(k_thomas_cyc<float>, THOMAS_BLOCK, thomas_cyc_smem<float>());
    cap[CAP_RM] = resident_grid(k_residmax, 256, 0);
    cap[CAP_RC] = resident_grid(k_resid_corr<true>, 256, 0);
    cap[CAP_CIF] = resident_grid(k_correct_if, 256, 0);
}

constexpr int kFluxKc = 32;  // planes marched by one flux CTA
dim3 flux_grid(int nx, int ny, int nz) {
    return dim3((nx + FLUX_BX - 1) / FLUX_BX, (ny + FLUX_BY - 1) / FLUX_BY, (nz + kFluxKc - 1) / kFluxKc);
}
size_t usq_blocks(const fizzy_proj_desc *d) {
    const dim3 gr = flux_grid(d->nx, d->ny, d->nz);
    return (size_t)gr.x * gr.y * gr.z;
}

size_t plan_bytes(const fizzy_proj_desc *d) {
    const size_t N = (size_t)d->nx * d->ny * d->nz;
    const int mixed = d->precision == FIZZY_PREC_MIXED;
    const size_t Ux = d->bc_x == FIZZY_BC_PERIODIC ? d->nx / 2 + 1 : d->nx;
    const size_t Uy = d->bc_y == FIZZY_BC_PERIODIC ? d->ny / 2 + 1 : d->ny;
    const size_t tab = Ux * Uy * d->nz;
    size_t b = 0;
    b += 3 * N * 8;                   // q
    b += mixed ? N * 4 + N * 8 : N * 8;  // spectral workspace (+ f in mixed)
    const size_t ntab = d->periodic_z ? 4 : 2;  // periodic z: + weights and correction vector
    b += ntab * tab * 8;              // FP64 factorisation tables
    if (mixed) b += ntab * tab * 4;   // FP32 factorisation tables
    b += 16 * (size_t)d->nz * 8;      // per-k tables
    b += 4 * (size_t)(d->nx + d->ny + 4) * 16;  // twiddles
    b += usq_blocks(d) * 8 + 4096;    // partials + stats
    return b;
}

// The probe kernel instance of an operation and chain count.
template <typename T> const void *probe_fn(int op, int chains) {
    const void *f[6][3] = {
        {(const void *)k_fma_probe<T, 0, 4>, (const void *)k_fma_probe<T, 0, 8>, (const void *)k_fma_probe<T, 0, 16>},
        {(const void *)k_fma_probe<T, 1, 4>, (const void *)k_fma_probe<T, 1, 8>, (const void *)k_fma_probe<T, 1, 16>},
        {(const void *)k_fma_probe<T, 2, 4>, (const void *)k_fma_probe<T, 2, 8>, (const void *)k_fma_probe<T, 2, 16>},
        {(const void *)k_fma_probe<T, 3, 4>, (const void *)k_fma_probe<T, 3, 8>, (const void *)k_fma_probe<T, 3, 16>},
        {(const void *)k_fma_probe<T, 4, 4>, (const void *)k_fma_probe<T, 4, 8>, (const void *)k_fma_probe<T, 4, 16>},
        {(const void *)k_fma_probe<T, 5, 4>, (const void *)k_fma_probe<T, 5, 8>, (const void *)k_fma_probe<T, 5, 16>}};
    return f[op][chains == 4 ? 0 : chains == 8 ? 1 : 2];
}

}  // namespace

extern "C" {

const char *fizzy_proj_errstr(int code) {
    if (code > 0 || code < -6) return "unknown error";
    return kErrStr[-code];
}

const char *fizzy_proj_last_error(fizzy_proj_plan_t p) { return p ? p->err.c_str() : ""; }

size_t fizzy_proj_workspace_bytes(const fizzy_proj_desc *d) {
    if (validate(d) != FIZZY_OK) return 0;
    return plan_bytes(d);
}

int fizzy_proj_destroy(fizzy_proj_plan_t p) {
    if (!p) return FIZZY_OK;
    if (p->async_alloc) {
        // stream-ordered: frees run after the work already queued on the plan's stream
        for (void *a : p->allocs) cudaFreeAsync(a, p->alloc_stream);
        if (p->arena) cudaFreeAsync(p->arena, p->alloc_stream);
        p->allocs.clear();
        p->arena = nullptr;
    } else {
        cudaDeviceSynchronize();
    }
    for (auto &e : p->ev) cudaEventDestroy(e);
    for (void *a : p->allocs) cudaFree(a);
    if (p->arena) cudaFree(p->arena);
    if (p->d2h) cudaStreamSynchronize(p->d2h);
    for (int b = 0; b < 2; ++b) {
        for (int t = 0; t < 7; ++t)
            if (p->stage[b][t]) cudaFree(p->stage[b][t]);
        for (cudaEvent_t e : {p->ev_in[b], p->ev_done[b], p->ev_out[b]})
            if (e) cudaEventDestroy(e);
    }
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    delete p;
    return FIZZY_OK;
}

int fizzy_proj_plan(fizzy_proj_plan_t *out, const fizzy_proj_desc *d, void *stream) {
    (void)stream;
    if (!out) return FIZZY_ERR_INVALID;
    *out = nullptr;
    int v = validate(d);
    if (v) return v;
    fizzy_proj_plan_s *p = new fizzy_proj_plan_s();
    p->desc = *d;
    p->async_alloc = (d->flags & FIZZY_FLAG_ASYNC_ALLOC) ? 1 : 0;
    p->alloc_stream = (cudaStream_t)stream;
    p->mixed = d->precision == FIZZY_PREC_MIXED;
    p->check = (d->flags & FIZZY_FLAG_CHECK) ? 1 : 0;
    p->tol = d->tol > 0 ? d->tol : 1e-10;
    p->max_refine = d->max_refine > 0 ? d->max_refine : FIZZY_DEFAULT_MAX_REFINE;
    p->div_tol = d->div_tol > 0 ? d->div_tol : (d->div_tol < 0 ? -1.0 : 1e-10);
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    const size_t N = (size_t)nx * ny * nz;
    p->zf.resize(nz + 1);
    for (int k = 0; k <= nz; ++k) p->zf[k] = d->zf ? d->zf[k] : d->dz * k;
    p->desc.zf = nullptr;

    // ---- grid metrics (host, FP64)
    std::vector<double> dzf(nz), zc(nz), dzc(nz, 0.0);
    for (int k = 0; k < nz; ++k) {
        dzf[k] = p->zf[k + 1] - p->zf[k];
        zc[k] = 0.5 * (p->zf[k] + p->zf[k + 1]);
    }
    for (int k = 0; k + 1 < nz; ++k) dzc[k] = zc[k + 1] - zc[k];
    const bool perz = d->periodic_z != 0;
    if (perz) dzc[nz - 1] = 0.5 * (dzf[0] + dzf[nz - 1]);  // the seam face nz-1/2
    double lz = 0.0;
    for (int k = 0; k < nz; ++k) lz += dzf[k];
    p->sigma = 1.0 / (4.0 * (double)nx * (double)ny);
    const double sig = p->sigma;
    // per-k tables, packed: T_NTAB arrays of nz (the physics rows first)
    enum { T_FAZ, T_FRZ, T_DVZ, T_DVZS, T_CGZ, T_LZA, T_LZC, T_IZF, T_DZF, T_DZC, T_NTAB };
    static_assert(T_LZA == kZPhys, "physics rows lead the per-k table block");
    std::vector<double> zt((size_t)T_NTAB * nz, 0.0);
    for (int k = 0; k < nz; ++k) {
        const bool top = (k == nz - 1) && !perz;
        physics_zrow(d->rho_l, d->rho_g, d->dt, sig, dzf[k], dzc[k], top, &zt[k], nz);
        zt[T_LZA * nz + k] = (k > 0) ? 1.0 / (dzf[k] * dzc[k - 1])
                                     : (perz ? 1.0 / (dzf[0] * dzc[nz - 1]) : 0.0);
        zt[T_LZC * nz + k] = top ? 0.0 : 1.0 / (dzf[k] * dzc[k]);  // periodic z: the seam at nz-1
        zt[T_IZF * nz + k] = 1.0 / dzf[k];
        zt[T_DZF * nz + k] = dzf[k];
        zt[T_DZC * nz + k] = dzc[k];
    }
    // the plan's device memory in one allocation (dev_alloc carves it)
    {
        p->arena_size = plan_bytes(d) + 64 * 256;
        void *a = nullptr;
        const cudaError_t e = p->async_alloc ? cudaMallocAsync(&a, p->arena_size, p->alloc_stream)
                                             : cudaMalloc(&a, p->arena_size);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            fizzy_proj_destroy(p);
            return FIZZY_ERR_NOMEM;
        }
        p->arena = (unsigned char *)a;
    }
    // eigenvalues of the x and y second differences per transform slot
    const int Ux = d->bc_x == FIZZY_BC_PERIODIC ? nx / 2 + 1 : nx;
    const int Uy = d->bc_y == FIZZY_BC_PERIODIC ? ny / 2 + 1 : ny;
    std::vector<double> lam((size_t)Ux + Uy);
    for (int u = 0; u < Ux; ++u) lam[u] = eig(u, nx, d->dx, d->bc_x);
    for (int u = 0; u < Uy; ++u) lam[Ux + u] = eig(u, ny, d->dy, d->bc_y);
    const double *C = &zt[T_LZC * nz];
    // one upload of the host-built tables: per-k rows | eigenvalues | c_k (FP64, FP32)
    const size_t o_lam = zt.size() * sizeof(double), o_c64 = o_lam + lam.size() * sizeof(double);
    const size_t o_c32 = o_c64 + (size_t)nz * sizeof(double), up_bytes = o_c32 + (size_t)nz * sizeof(float);
    int status = 0;
    unsigned char *up_d = dev_alloc<unsigned char>(p, up_bytes, &status);
    if (status) {
        int st = status;
        fizzy_proj_destroy(p);
        return st;
    }
    {
        std::vector<unsigned char> up(up_bytes);
        memcpy(up.data(), zt.data(), o_lam);
        memcpy(up.data() + o_lam, lam.data(), lam.size() * sizeof(double));
        memcpy(up.data() + o_c64, C, (size_t)nz * sizeof(double));
        for (int k = 0; k < nz; ++k) {
            const float c = (float)C[k];
            memcpy(up.data() + o_c32 + (size_t)k * sizeof(float), &c, sizeof(float));
        }
        note(p, cudaMemcpyAsync(up_d, up.data(), up_bytes, cudaMemcpyHostToDevice, p->alloc_stream));
    }
    double *zt_d = (double *)up_d;
    const double *lam_d = (const double *)(up_d + o_lam);
    p->zt = zt_d;
    p->cup64 = (double *)(up_d + o_c64);
    p->cup32 = p->mixed ? (float *)(up_d + o_c32) : nullptr;

    GridDev &g = p->g;
    memset(&g, 0, sizeof(g));
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.bcx = d->bc_x;
    g.bcy = d->bc_y;
    g.perz = d->periodic_z ? 1 : 0;
    g.sing = (d->bc_x <= FIZZY_BC_NEUMANN && d->bc_y <= FIZZY_BC_NEUMANN) ? 1 : 0;
    g.rny = (unsigned)((1ull << 32) / (unsigned)ny + 1);
    physics_consts(g, d->rho_l, d->rho_g, d->dt, d->dx, d->dy, sig);
    g.flux_df = p->mixed;
    g.idx2 = 1.0 / (d->dx * d->dx);
    g.idy2 = 1.0 / (d->dy * d->dy);
    g.idx1 = 1.0 / d->dx;
    g.idy1 = 1.0 / d->dy;
    g.faz = zt_d + T_FAZ * nz;
    g.frz = zt_d + T_FRZ * nz;
    g.dvz = zt_d + T_DVZ * nz;
    g.dvz_s = zt_d + T_DVZS * nz;
    g.cgz = zt_d + T_CGZ * nz;
    g.lza = zt_d + T_LZA * nz;
    g.lzc = zt_d + T_LZC * nz;
    g.izf = zt_d + T_IZF * nz;
    g.dzf = zt_d + T_DZF * nz;
    g.dzc = zt_d + T_DZC * nz;
    g.inv_lz = 1.0 / lz;
    g.sigma = sig;
    g.inv_3n = 1.0 / (3.0 * (double)N);
    g.div_tol = p->div_tol;

    // ---- transforms
    build_fft(p, nx, d->bc_x, p->fx, &status);
    build_fft(p, ny, d->bc_y, p->fy, &status);

    // ---- z factorisation tables per distinct eigenvalue pair
    p->Ux = Ux;
    p->Uy = Uy;
    const size_t ts = (size_t)Ux * Uy;
    p->mtab64 = dev_alloc<double>(p, ts * nz, &status);
    p->ibtab64 = dev_alloc<double>(p, ts * nz, &status);
    if (p->mixed) {
        p->mtab32 = dev_alloc<float>(p, ts * nz, &status);
        p->ibtab32 = dev_alloc<float>(p, ts * nz, &status);
    }
    if (perz) {
        p->wtab64 = dev_alloc<double>(p, ts * nz, &status);
        p->qtab64 = dev_alloc<double>(p, ts * nz, &status);
        if (p->mixed) {
            p->wtab32 = dev_alloc<float>(p, ts * nz, &status);
            p->qtab32 = dev_alloc<float>(p, ts * nz, &status);
        }
    }
    // ---- workspace
    p->qx = dev_alloc<double>(p, N, &status);
    p->qy = dev_alloc<double>(p, N, &status);
    p->qz = dev_alloc<double>(p, N, &status);
    if (p->mixed) {
        p->fhat32 = dev_alloc<float>(p, N, &status);
        p->f = dev_alloc<double>(p, N, &status);
    } else {
        p->fhat64 = dev_alloc<double>(p, N, &status);
    }
    p->st = dev_alloc<DevStats>(p, 1, &status);
    p->n_usq_part = (int)usq_blocks(d);
    p->usq_part = dev_alloc<double>(p, p->n_usq_part, &status);
    p->usq_sum = dev_alloc<double>(p, 1, &status);
    p->g.usq = p->usq_sum;
    if (status) {
        int st = status;
        fizzy_proj_destroy(p);
        return st;
    }
    // factorisation tables on the device (bitwise the host recurrence)
    {
        const int blocks = (int)std::min<size_t>((ts + 127) / 128, 4096);
        if (perz)
            k_ztables_cyc<<<blocks, 128, 0, p->alloc_stream>>>(
                Ux, Uy, nz, lam_d, lam_d + Ux, zt_d + T_LZA * nz, zt_d + T_LZC * nz, p->mtab64,
                p->ibtab64, p->wtab64, p->qtab64, p->mixed ? p->mtab32 : nullptr,
                p->mixed ? p->ibtab32 : nullptr, p->mixed ? p->wtab32 : nullptr,
                p->mixed ? p->qtab32 : nullptr, g.sing);
        else
            k_ztables<<<blocks, 128, 0, p->alloc_stream>>>(Ux, Uy, nz, lam_d, lam_d + Ux, zt_d + T_LZA * nz,
                                                           zt_d + T_LZC * nz, p->mtab64, p->ibtab64,
                                                           p->mixed ? p->mtab32 : nullptr,
                                                           p->mixed ? p->ibtab32 : nullptr, g.sing);
    }
    note(p, cudaMemsetAsync(p->st, 0, sizeof(DevStats), p->alloc_stream));

    // ---- launch shapes and shared-memory opt-in
    p->Lx = x_lines_per_cta(nx);
    // mixed plans with a direction of length 128 to 512 (periodic or walls)
    // run the register-resident FP32 passes along it: static shared memory only
    const bool y_r16 = p->mixed && r_len(ny) != 0 && d->bc_y <= FIZZY_BC_NEUMANN;
    p->x_r16 = p->mixed && r_len(nx) != 0 && d->bc_x <= FIZZY_BC_NEUMANN;
    p->TXy = y_r16 ? r_tile_cols(ny) : y_tile_cols(ny, p->mixed != 0);
    p->smem_x64 = pass_smem<double>(nx, p->Lx);
    p->smem_x32 = pass_smem<float>(nx, p->Lx);
    p->smem_y64 = pass_smem<double>(ny, p->TXy / 2);
    p->smem_y32 = y_r16 ? 0 : pass_smem<float>(ny, p->TXy / 2);
    {  // opt-in shared-memory limits, once per device (plans may be built concurrently)
        static std::mutex attrs_mu;
        static bool attrs_set[256] = {false};
        int cur_dev = 0;
        note(p, cudaGetDevice(&cur_dev));
        std::lock_guard<std::mutex> lock(attrs_mu);
        if (cur_dev < 0 || cur_dev >= 256 || !attrs_set[cur_dev]) {
            if (cur_dev >= 0 && cur_dev < 256) attrs_set[cur_dev] = true;
            opt_in_smem(p, 200 * 1024);
        }
    }
    p->kern = pick_kernels(fixed_len(nx, d->bc_x), fixed_len(ny, d->bc_y));
    if (p->mixed) pick_r_kernels(p->kern, p->x_r16 ? nx : 0, d->bc_x, y_r16 ? ny : 0, d->bc_y);
    if (p->mixed && p->x_r16 && y_r16 && nx == ny && (nx == 256 || nx == 512) &&
        (d->flags & FIZZY_FLAG_FUSED_XY))
        p->xy_fused = setup_xy(p, nx, d->bc_x == FIZZY_BC_NEUMANN ? KIND_DCT : KIND_PERIODIC,
                               d->bc_y == FIZZY_BC_NEUMANN ? KIND_DCT : KIND_PERIODIC);
    p->xthr32 = p->x_r16 ? r_threads(nx) : 256;
    p->ythr32 = y_r16 ? r_threads(ny) : 256;
    pass_caps(p->cap, p->kern, p->smem_x64, p->smem_x32, p->x_r16 ? 0 : p->smem_x32, p->smem_y64,
              p->smem_y32, p->xthr32, p->ythr32);
    // stream-ordered plans are ready for work queued after them on their
    // stream; other plans are complete on return
    cudaError_t e = p->async_alloc ? cudaGetLastError() : cudaDeviceSynchronize();
    if (e == cudaSuccess) e = p->setup_err;
    if (e != cudaSuccess) {
        int st = cuda_err(nullptr, e, "plan");
        fizzy_proj_destroy(p);
        return st;
    }
    *out = p;
    return FIZZY_OK;
}

int fizzy_proj_set_physics(fizzy_proj_plan_t p, double rho_l, double rho_g, double dt, void *stream) {
    if (!p) return FIZZY_ERR_INVALID;
    if (!(rho_l >= 1e-30 && rho_l <= 1e30) || !(rho_g >= 1e-30 && rho_g <= 1e30) || !(dt > 0) ||
        !std::isfinite(dt))
        return set_err(p, FIZZY_ERR_INVALID, "bad densities or dt");
    const int nx = p->desc.nx, ny = p->desc.ny, nz = p->desc.nz;
    const double dx = p->desc.dx, dy = p->desc.dy;
    const double sig = p->sigma;
    // the physics rows of the per-k tables (see fizzy_proj_plan)
    std::vector<double> rows(kZPhys * (size_t)nz);
    for (int k = 0; k < nz; ++k) {
        const double dzf = p->zf[k + 1] - p->zf[k];
        const bool last = (k == nz - 1), top = last && !p->g.perz;
        const double zc0 = 0.5 * (p->zf[k] + p->zf[k + 1]);
        const double dzc = top ? 0.0
                           : last ? 0.5 * ((p->zf[1] - p->zf[0]) + dzf)  // periodic z: the seam
                                  : 0.5 * (p->zf[k + 1] + p->zf[k + 2]) - zc0;
        physics_zrow(rho_l, rho_g, dt, sig, dzf, dzc, top, &rows[k], nz);
    }
    const cudaError_t e = cudaMemcpyAsync(p->zt, rows.data(), rows.size() * sizeof(double),
                                          cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(p, e, "set_physics");
    physics_consts(p->g, rho_l, rho_g, dt, dx, dy, sig);
    p->desc.rho_l = rho_l;
    p->desc.rho_g = rho_g;
    p->desc.dt = dt;
    (void)nx;
    (void)ny;
    return FIZZY_OK;
}

int fizzy_proj_launches_per_solve(fizzy_proj_plan_t p) {
    if (!p) return 0;
    int n = p->mixed ? (p->xy_fused ? 7 + 4 * p->max_refine : 9 + 6 * p->max_refine) : 7;
    if (p->check) n += p->mixed ? 1 : 3;
    return n;
}

static void read_stats(fizzy_proj_plan_t p, const DevStats &h, double usq, fizzy_proj_stats *st) {
    memset(st, 0, sizeof(*st));
    const size_t N = (size_t)p->desc.nx * p->desc.ny * p->desc.nz;
    st->iterations = p->mixed ? h.iterations : 0;
    st->converged = p->mixed ? h.converged : 1;
    st->relres = h.relres;
    memcpy(&st->f_max, &h.fmax_bits, sizeof(double));
    memcpy(&st->div_max, &h.divmax_bits, sizeof(double));
    st->u_rms = (p->check || p->mixed) ? std::sqrt(usq / (3.0 * (double)N)) : 0.0;
    st->div_metric = (p->check && st->u_rms > 0) ? st->div_max * p->desc.dx / st->u_rms : 0.0;
}

int fizzy_proj_get_stats(fizzy_proj_plan_t p, fizzy_proj_stats *st, void *stream) {
    if (!p || !st) return FIZZY_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    DevStats h;
    double usq = 0.0;
    cudaError_t e = cudaMemcpyAsync(&h, p->st, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && (p->check || p->mixed))
        e = cudaMemcpyAsync(&usq, p->usq_sum, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(p, e, "get_stats");
    read_stats(p, h, usq, st);
    if (p->mixed && !st->converged) return FIZZY_ERR_NOT_CONVERGED;
    return FIZZY_OK;
}

static inline void tmark(fizzy_proj_plan_t p, int slot, cudaStream_t s, bool begin) {
    if (!p->timing || (p->timing >= 2 && slot != p->timing - 2)) return;
    if (begin) {
        if (p->ev_used >= kMaxTimed) return;
        cudaEventRecord(p->ev[2 * p->ev_used], s);
        p->ev_slot[p->ev_used] = slot;
    } else {
        if (p->ev_used >= kMaxTimed || p->ev_slot[p->ev_used] != slot) return;
        cudaEventRecord(p->ev[2 * p->ev_used + 1], s);
        ++p->ev_used;
    }
}
#define TIMED(slot, launch)          \
    do {                             \
        tmark(p, slot, s, true);     \
        launch;                      \
        tmark(p, slot, s, false);    \
    } while (0)

int fizzy_proj_set_timing(fizzy_proj_plan_t p, int enable) {
    if (!p || enable < 0 || enable >= 2 + KS_N) return FIZZY_ERR_INVALID;
    if (enable && p->ev.empty()) {
        p->ev.resize(2 * kMaxTimed);
        p->ev_slot.assign(kMaxTimed, -1);
        for (auto &e : p->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return cuda_err(p, r, "event create");
        }
    }
    p->timing = enable;
    p->ev_used = 0;
    for (int k = 0; k < KS_N; ++k) {
        p->t_ms[k] = 0.0;
        p->t_cnt[k] = 0;
    }
    return FIZZY_OK;
}

int fizzy_proj_timing(fizzy_proj_plan_t p, int idx, const char **name, double *ms, int *launches) {
    if (!p) return FIZZY_ERR_INVALID;
    for (int t = 0; t < p->ev_used; ++t) {
        cudaError_t r = cudaEventSynchronize(p->ev[2 * t + 1]);
        if (r != cudaSuccess) return cuda_err(p, r, "event sync");
        float e = 0.f;
        cudaEventElapsedTime(&e, p->ev[2 * t], p->ev[2 * t + 1]);
        p->t_ms[p->ev_slot[t]] += e;
        p->t_cnt[p->ev_slot[t]] += 1;
    }
    p->ev_used = 0;
    if (idx >= 0 && idx < KS_N) {
        if (name) *name = kSlotName[idx];
        if (ms) *ms = p->t_ms[idx];
        if (launches) *launches = p->t_cnt[idx];
    }
    return KS_N;
}

// The launches of one solve.  sw_first = 0: the whole sequence with the
// refinement sweeps 1 .. sw_last (mixed) and the conditional correction;
// sw_first >= 1 (mixed only): the sweeps sw_first .. sw_last alone, which
// continue a solve whose sweeps up to sw_first - 1 ran without converging
// (the stored residual, p and u are where those sweeps left them).  The
// kernels of a sweep return at once when the solve has converged, so the
// results do not depend on how the sweeps are split between calls.
static int solve_launch(fizzy_proj_plan_t p, const double *phi, const double *p_n,
                        const double *p_nm1, double *u, double *v, double *w, double *p_np1,
                        cudaStream_t s, int sw_first, int sw_last);

int fizzy_proj_solve(fizzy_proj_plan_t p, const double *phi, const double *p_n, const double *p_nm1,
                     double *u, double *v, double *w, double *p_np1, fizzy_proj_stats *st,
                     void *stream) {
    if (!p) return FIZZY_ERR_INVALID;
    const int rc = solve_launch(p, phi, p_n, p_nm1, u, v, w, p_np1, (cudaStream_t)stream, 0, p->max_refine);
    if (rc) return rc;
    if (st) return fizzy_proj_get_stats(p, st, stream);
    return FIZZY_OK;
}

static int solve_launch(fizzy_proj_plan_t p, const double *phi, const double *p_n,
                        const double *p_nm1, double *u, double *v, double *w, double *p_np1,
                        cudaStream_t s, int sw_first, int sw_last) {
    if (!phi || !p_n || !p_nm1 || !u || !v || !w || !p_np1)
        return set_err(p, FIZZY_ERR_INVALID, "null array pointer");
    if (p_np1 == phi || p_np1 == p_n || p_np1 == p_nm1 || p_np1 == u || p_np1 == v || p_np1 == w)
        return set_err(p, FIZZY_ERR_INVALID, "p_np1 aliases an input");
    if (!staggered_bcs(p->desc)) return set_err(p, FIZZY_ERR_UNSUPPORTED, kNeedsStaggeredBcs);
    if (sw_first < 0 || (sw_first > 0 && !p->mixed) || sw_last > p->max_refine)
        return set_err(p, FIZZY_ERR_INVALID, "refinement sweeps out of range");
    const bool head = sw_first == 0;  // the sequence up to the residual of the FP32 solution
    const GridDev &g = p->g;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const dim3 cblk(32, 8), cgrd((nx + 31) / 32, (ny + 7) / 8, nz);
    const dim3 rblk(256), rgrd((nx + 255) / 256, ny, nz);
    const int nlines = ny * nz;
    // tiles of each pass; each stand-alone launch runs min(tiles, resident grid)
    const int xtiles = (nlines + 2 * p->Lx - 1) / (2 * p->Lx);
    // the FP32 x-passes: 32 (n = 256) or 16 (n = 512) lines per tile when
    // register-resident
    const int xrt = p->x_r16 ? (nlines + r_tile_lines(nx) - 1) / r_tile_lines(nx) : xtiles;
    const size_t smx32r = p->x_r16 ? 0 : p->smem_x32;
    const int ygx = (nx + p->TXy - 1) / p->TXy, ytiles = ygx * nz;
    const int ttiles = (nx * ny + THOMAS_BLOCK - 1) / THOMAS_BLOCK;  // one z-line per thread
    const int rgx = (nx + 255) / 256, rtiles = rgx * ny * nz;
    // main path: one block per tile; refinement passes that usually find the
    // solve converged, and the final check: the resident grid
    auto grid = [&](int tiles, int) { return std::max(1, tiles); };
    auto rgrid = [&](int tiles, int c) { return std::max(1, std::min(tiles, p->cap[c])); };
    XArgs xa;
    memset(&xa, 0, sizeof(xa));
    xa.qx = p->qx;
    xa.qy = p->qy;
    xa.qz = p->qz;
    xa.st = p->st;
    cudaError_t e = cudaSuccess;
    if (head && (p->mixed || p->check)) e = cudaMemsetAsync(p->st, 0, sizeof(DevStats), s);
    if (e != cudaSuccess) return cuda_err(p, e, "memset");

    const bool need_usq = p->check || p->mixed;
    const dim3 fgrd = flux_grid(nx, ny, nz), fblk(FLUX_BX, FLUX_BY);
    if (!head) {
        // continuation: only the sweeps below
    } else {
        const bool g0 = p->desc.rho_g <= p->desc.rho_l;
        auto kf = g.flux_df ? (g0 ? k_flux_df<true> : k_flux_df<false>) : (g0 ? k_flux<true> : k_flux<false>);
        TIMED(KS_FLUX, (kf<<<fgrd, fblk, 0, s>>>(g, kFluxKc, phi, p_n, p_nm1, u, v, w, p->qx, p->qy, p->qz,
                                                 need_usq ? p->usq_part : nullptr)));
    }
    if (head && need_usq)
        TIMED(KS_SUM, (k_sum_partials<<<1, 1024, 0, s>>>(p->usq_part, p->n_usq_part, p->usq_sum)));
    if (!p->mixed) {
        xa.out = p->fhat64;
        TIMED(KS_XFWD, (p->kern.xf64<<<grid(xtiles, CAP_XF64), 256, p->smem_x64, s>>>(g, p->fx.d64, p->Lx, xa, xtiles)));
        TIMED(KS_YFWD, (p->kern.yf64<<<grid(ytiles, CAP_Y64F), 256, p->smem_y64, s>>>(nx, ny, p->fy.d64, p->TXy, p->fhat64, nullptr, ygx, ytiles)));
        if (g.perz)
            TIMED(KS_THOMAS, (k_thomas_cyc<double><<<grid(ttiles, CAP_TH64C), THOMAS_BLOCK, thomas_cyc_smem<double>(), s>>>(g, p->Ux, p->Uy, p->mtab64, p->ibtab64, p->cup64, p->wtab64, p->qtab64, p->fhat64, nullptr, ttiles)));
        else
            TIMED(KS_THOMAS, (k_thomas<double><<<grid(ttiles, CAP_TH64), THOMAS_BLOCK, thomas_smem<double>(), s>>>(g, p->Ux, p->Uy, p->mtab64, p->ibtab64, p->cup64, p->fhat64, nullptr, ttiles)));
        TIMED(KS_YINV, (p->kern.yi64<<<grid(ytiles, CAP_Y64I), 256, p->smem_y64, s>>>(nx, ny, p->fy.d64, p->TXy, p->fhat64, nullptr, ygx, ytiles)));
        TIMED(KS_XINV, (p->kern.xi64<<<grid(xtiles, CAP_XI64), 256, p->smem_x64, s>>>(g, p->fx.d64, p->Lx, p->fhat64, p_np1, p->st, xtiles)));
        if (p->check) {
            XArgs ca = xa;
            ca.p = p_np1;
            TIMED(KS_RESMAX, (k_residmax<<<grid(rtiles, CAP_RM), rblk, 0, s>>>(g, ca, rgx, rtiles)));
        }
    } else {
        xa.out = p->fhat32;
        xa.f_out = p->f;
        const int *conv = &p->st->converged;
        const int xyg = XY_CL * nz;  // fused x-y passes: one cluster per z-plane
        if (!head) {
            // continuation: the FP32 solution, its residual and the first
            // sweeps are already on the stream
        } else if (p->xy_fused) {
            TIMED(KS_XFWD, (p->xyf_div<<<xyg, p->xy_threads, p->xy_smem, s>>>(g, xa)));
        } else {
            TIMED(KS_XFWD, (p->kern.xf32d<<<grid(xrt, CAP_XF32D), p->xthr32, smx32r, s>>>(g, p->fx.d32, p->Lx, xa, xrt)));
            TIMED(KS_YFWD, (p->kern.yf32<<<grid(ytiles, CAP_Y32F), p->ythr32, p->smem_y32, s>>>(nx, ny, p->fy.d32, p->TXy, p->fhat32, nullptr, ygx, ytiles)));
        }
        if (head) {
            if (g.perz)
                TIMED(KS_THOMAS, (k_thomas_cyc<float><<<grid(ttiles, CAP_TH32C), THOMAS_BLOCK, thomas_cyc_smem<float>(), s>>>(g, p->Ux, p->Uy, p->mtab32, p->ibtab32, p->cup32, p->wtab32, p->qtab32, p->fhat32, nullptr, ttiles)));
            else
                TIMED(KS_THOMAS, (k_thomas<float><<<grid(ttiles, CAP_TH32), THOMAS_BLOCK, thomas_smem<float>(), s>>>(g, p->Ux, p->Uy, p->mtab32, p->ibtab32, p->cup32, p->fhat32, nullptr, ttiles)));
        }
        if (!head) {
        } else if (p->xy_fused) {
            TIMED(KS_XINV, (p->xyi_store<<<xyg, p->xy_threads, p->xy_smem, s>>>(g, p->fhat32, p_np1, p->st)));
        } else {
            TIMED(KS_YINV, (p->kern.yi32<<<grid(ytiles, CAP_Y32I), p->ythr32, p->smem_y32, s>>>(nx, ny, p->fy.d32, p->TXy, p->fhat32, nullptr, ygx, ytiles)));
            TIMED(KS_XINV, (p->kern.xi32s<<<grid(xrt, CAP_XI32S), p->xthr32, smx32r, s>>>(g, p->fx.d32, p->Lx, p->fhat32, p_np1, p->st, xrt)));
        }
        // residual of the FP32 solution (slot 0), then refinement sweeps
        // sw = 1..max_refine: transform of the stored residual, FP32 y/z/y^-1,
        // p += delta, then the residual fused with the correction (slot sw)
        RArgs ra;
        ra.p = p_np1;
        ra.f = p->f;
        ra.qx = p->qx;
        ra.qy = p->qy;
        ra.qz = p->qz;
        ra.u = u;
        ra.v = v;
        ra.w = w;
        ra.r32 = p->fhat32;
        ra.st = p->st;
        ra.tol = p->tol;
        ra.slot = 0;
        const dim3 rcb(FLUX_BX, FLUX_BY);
        const int rtgx = (nx + FLUX_BX - 1) / FLUX_BX, rtgy = (ny + FLUX_BY - 1) / FLUX_BY;
        const int rctiles = rtgx * rtgy * ((nz + RESID_KC - 1) / RESID_KC);
        if (head)
            TIMED(KS_RESID, (k_resid<false><<<grid(rctiles, CAP_RC), rcb, 0, s>>>(g, RESID_KC, ra, rtgx, rtgy, rctiles)));
        XArgs la = xa;  // in-place transform of the stored residual
        la.f_out = nullptr;
        const int sw0 = head ? 1 : sw_first;
        for (int sw = sw0; sw <= sw_last; ++sw) {
            // the first sweep of a call runs a grid per tile; later sweeps
            // usually return at once and run the resident grid
            auto gs = [&](int tiles, int c) { return sw == sw0 ? grid(tiles, c) : rgrid(tiles, c); };
            if (p->xy_fused) {
                TIMED(KS_XFWD_R, (p->xyf_load<<<xyg, p->xy_threads, p->xy_smem, s>>>(g, la)));
            } else {
                TIMED(KS_XFWD_R, (p->kern.xf32l<<<gs(xrt, CAP_XF32L), p->xthr32, smx32r, s>>>(g, p->fx.d32, p->Lx, la, xrt)));
                TIMED(KS_YFWD_R, (p->kern.yf32<<<gs(ytiles, CAP_Y32F), p->ythr32, p->smem_y32, s>>>(nx, ny, p->fy.d32, p->TXy, p->fhat32, conv, ygx, ytiles)));
            }
            if (g.perz)
                TIMED(KS_THOMAS_R, (k_thomas_cyc<float><<<gs(ttiles, CAP_TH32C), THOMAS_BLOCK, thomas_cyc_smem<float>(), s>>>(g, p->Ux, p->Uy, p->mtab32, p->ibtab32, p->cup32, p->wtab32, p->qtab32, p->fhat32, conv, ttiles)));
            else
                TIMED(KS_THOMAS_R, (k_thomas<float><<<gs(ttiles, CAP_TH32), THOMAS_BLOCK, thomas_smem<float>(), s>>>(g, p->Ux, p->Uy, p->mtab32, p->ibtab32, p->cup32, p->fhat32, conv, ttiles)));
            if (p->xy_fused) {
                TIMED(KS_XACC, (p->xyi_accum<<<xyg, p->xy_threads, p->xy_smem, s>>>(g, p->fhat32, p_np1, p->st)));
            } else {
                TIMED(KS_YINV_R, (p->kern.yi32<<<gs(ytiles, CAP_Y32I), p->ythr32, p->smem_y32, s>>>(nx, ny, p->fy.d32, p->TXy, p->fhat32, conv, ygx, ytiles)));
                TIMED(KS_XACC, (p->kern.xi32a<<<gs(xrt, CAP_XI32A), p->xthr32, smx32r, s>>>(g, p->fx.d32, p->Lx, p->fhat32, p_np1, p->st, xrt)));
            }
            ra.slot = sw;
            TIMED(KS_RCORR, (k_resid_corr<true><<<gs(rctiles, CAP_RC), rcb, 0, s>>>(g, RESID_KC, ra, rtgx, rtgy, rctiles)));
        }
        // the correction, unless a fused residual pass has written u (a
        // continuation follows at least one fused pass: nothing to do)
        const int ctiles = rtgx * rtgy * nz;
        if (head)
            TIMED(KS_CORRECT, (k_correct_if<<<rgrid(ctiles, CAP_CIF), rcb, 0, s>>>(g, p_np1, p->qx, p->qy, p->qz, u, v, w, p->st, rtgx, rtgy, ctiles)));
    }
    if (!p->mixed) TIMED(KS_CORRECT, (k_correct<<<cgrd, cblk, 0, s>>>(g, p_np1, p->qx, p->qy, p->qz, u, v, w)));
    if (p->check && !head) {  // the continuation's u replaces the one measured before
        e = cudaMemsetAsync(&p->st->divmax_bits, 0, sizeof(p->st->divmax_bits), s);
        if (e != cudaSuccess) return cuda_err(p, e, "memset");
    }
    if (p->check) TIMED(KS_DIVMAX, (k_divmax<<<rgrd, rblk, 0, s>>>(g, u, v, w, p->st)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(p, e, "solve launch");
    return FIZZY_OK;
}

// Staging for the host-array entry points: both sets, the copy streams and
// the events, made once.
static int host_staging(fizzy_proj_plan_t p) {
    if (p->h2d) return FIZZY_OK;
    const size_t B = (size_t)p->desc.nx * p->desc.ny * p->desc.nz * sizeof(double);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        for (int t = 0; t < 7 && e == cudaSuccess; ++t) e = cudaMalloc(&p->stage[b][t], B);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        for (int b = 0; b < 2; ++b)
            for (int t = 0; t < 7; ++t) {
                if (p->stage[b][t]) cudaFree(p->stage[b][t]);
                p->stage[b][t] = nullptr;
            }
        return set_err(p, FIZZY_ERR_NOMEM, "staging allocation failed");
    }
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&p->ev_in[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_out[b], cudaEventDisableTiming);
    }
    cudaStream_t h2d = nullptr, d2h = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (h2d) cudaStreamDestroy(h2d);
        return cuda_err(p, e, "staging streams");
    }
    p->h2d = h2d;
    p->d2h = d2h;
    return FIZZY_OK;
}

int fizzy_proj_solve_host_async(fizzy_proj_plan_t p, const double *phi, const double *p_n,
                                const double *p_nm1, const double *u_in, const double *v_in,
                                const double *w_in, double *u, double *v, double *w, double *p_np1,
                                void *stream) {
    if (!p) return FIZZY_ERR_INVALID;
    if (!phi || !p_n || !p_nm1 || !u_in || !v_in || !w_in || !u || !v || !w || !p_np1)
        return set_err(p, FIZZY_ERR_INVALID, "null array pointer");
    if (!staggered_bcs(p->desc)) return set_err(p, FIZZY_ERR_UNSUPPORTED, kNeedsStaggeredBcs);
    int rc = host_staging(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t B = (size_t)p->desc.nx * p->desc.ny * p->desc.nz * sizeof(double);
    const int b = p->host_calls & 1;
    double *const *d = p->stage[b];
    // 1. inputs into set b, once its previous results have been copied out
    cudaError_t e = p->set_used[b] ? cudaStreamWaitEvent(p->h2d, p->ev_out[b], 0) : cudaSuccess;
    const double *hin[6] = {phi, p_n, p_nm1, u_in, v_in, w_in};
    for (int t = 0; t < 6 && e == cudaSuccess; ++t)
        e = cudaMemcpyAsync(d[t], hin[t], B, cudaMemcpyHostToDevice, p->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[b], p->h2d);
    // 2. the solve on the caller's stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_in[b], 0);
    if (e != cudaSuccess) return cuda_err(p, e, "H2D");
    rc = fizzy_proj_solve(p, d[0], d[1], d[2], d[3], d[4], d[5], d[6], nullptr, stream);
    if (rc) return rc;
    e = cudaEventRecord(p->ev_done[b], s);
    // 3. results back
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_done[b], 0);
    double *hout[4] = {u, v, w, p_np1};
    const int src[4] = {3, 4, 5, 6};
    for (int t = 0; t < 4 && e == cudaSuccess; ++t)
        e = cudaMemcpyAsync(hout[t], d[src[t]], B, cudaMemcpyDeviceToHost, p->d2h);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_out[b], p->d2h);
    if (e != cudaSuccess) return cuda_err(p, e, "D2H");
    p->set_used[b] = true;
    ++p->host_calls;
    return FIZZY_OK;
}


int fizzy_probe_fma_rate(int precision, int op, int chains, int iters, double *instr_per_s,
                         double *elapsed_ms, void *stream) {
    if (iters < 1 || !instr_per_s || op < 0 || op > 5 || (chains != 4 && chains != 8 && chains != 16))
        return FIZZY_ERR_INVALID;
    if (precision != FIZZY_PREC_FP64 && precision != FIZZY_PREC_MIXED) return FIZZY_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const bool f64 = precision == FIZZY_PREC_FP64;
    const void *fn = f64 ? probe_fn<double>(op, chains) : probe_fn<float>(op, chains);
    int dev = 0, sms = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, 0);
    if (e != cudaSuccess) return FIZZY_ERR_CUDA;
    const int grid = std::max(1, nb) * std::max(1, sms);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        double a64 = 0.9999999, b64 = 1e-7;
        float a32 = 0.9999f, b32 = 1e-4f;
        void *args64[] = {&iters, &a64, &b64};
        void *args32[] = {&iters, &a32, &b32};
        e = cudaLaunchKernel(fn, dim3(grid), dim3(256), f64 ? args64 : args32, 0, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.f)) return FIZZY_ERR_CUDA;
    const double instr = (double)grid * 256.0 * (double)iters * 4.0 * chains;
    *instr_per_s = instr / (ms * 1e-3);
    if (elapsed_ms) *elapsed_ms = ms;
    return FIZZY_OK;
}

int fizzy_proj_host_wait(fizzy_proj_plan_t p) {
    if (!p) return FIZZY_ERR_INVALID;
    if (!p->d2h) return FIZZY_OK;
    const cudaError_t e = cudaStreamSynchronize(p->d2h);
    if (e != cudaSuccess) return cuda_err(p, e, "host wait");
    return FIZZY_OK;
}

int fizzy_proj_solve_host(fizzy_proj_plan_t p, const double *phi, const double *p_n,
                          const double *p_nm1, double *u, double *v, double *w, double *p_np1,
                          fizzy_proj_stats *st, void *stream) {
    int rc = fizzy_proj_solve_host_async(p, phi, p_n, p_nm1, u, v, w, u, v, w, p_np1, stream);
    if (rc == FIZZY_OK) rc = fizzy_proj_host_wait(p);
    if (rc) return rc;
    if (st) return fizzy_proj_get_stats(p, st, stream);
    return FIZZY_OK;
}

}  // extern "C"

// ===========================================================================
// Stand-alone Poisson solve with every boundary kind (fizzy_poisson_solve)
// ===========================================================================
#include "fizzy_poisson.inc"

// ===========================================================================
// Batched projections (fizzy_proj_batch_*)
// ===========================================================================
#include "fizzy_batch.inc"

// ===========================================================================
// Variable-coefficient projection without splitting (fizzy_proj_solve_vc)
// ===========================================================================
#include "fizzy_vc.inc"

// ===========================================================================
// ACDI phase-field step (fizzy_acdi_step)
// ===========================================================================
#include "fizzy_acdi.inc"

// ===========================================================================
// Serving runtime (fizzy_serve_*)
// ===========================================================================
#include "fizzy_serve.inc"

// ===========================================================================
// Allocation-free projection (fizzy_proj_solve_noalloc): the FP64 kernel
// sequence of fizzy_proj_solve on tables and workspace kept in one static
// device array, for callers that cannot allocate device memory.
// ===========================================================================
namespace {

constexpr int kNaMaxCells = FIZZY_NOALLOC_MAX_CELLS;
constexpr int kNaMaxN = 512;
constexpr int kNaMaxNz = 4096;
constexpr int kNaZTabs = 10;  // per-k tables, in the order of the plan's T_* enum
// layout in doubles: q (3N) | fhat (N) | m table (N) | 1/beta table (N) |
// per-k tables (10 x nz) | upper z coefficient (nz) | x twiddles | x cos/sin |
// y twiddles | y cos/sin
constexpr size_t kNaTw = 2 * (size_t)kNaMaxN;
constexpr size_t kNaCs = 2 * (size_t)(kNaMaxN / 2 + 2);
constexpr size_t kNaDoubles = 6 * (size_t)kNaMaxCells + (kNaZTabs + 1) * (size_t)kNaMaxNz +
                              2 * (kNaTw + kNaCs) + 32;
static_assert(kNaDoubles * sizeof(double) == FIZZY_NOALLOC_SCRATCH_BYTES,
              "header scratch size out of date");

// The scratch: shared by every call on a device, held until process exit.
static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];
// Host-side staging of the tables (also shared by all calls).
static double g_noalloc_host[2 * (size_t)kNaMaxCells + (kNaZTabs + 1) * (size_t)kNaMaxNz +
                            2 * (kNaTw + kNaCs)];
// Device address of the scratch per device ordinal (0 = not looked up yet).
static double *g_noalloc_dev[256];

}  // namespace

extern "C" int fizzy_proj_solve_noalloc(const fizzy_proj_desc *d, const double *phi,
                                        const double *p_n, const double *p_nm1, double *u,
                                        double *v, double *w, double *p_np1, void *stream) {
    const int vrc = validate(d);
    if (vrc) return vrc;
    if (!phi || !p_n || !p_nm1 || !u || !v || !w || !p_np1) return FIZZY_ERR_INVALID;
    if (d->precision != FIZZY_PREC_FP64 || d->flags != 0) return FIZZY_ERR_INVALID;
    if (d->periodic_z || !staggered_bcs(*d)) return FIZZY_ERR_UNSUPPORTED;  // walls in z; P/N x, y
    const int nx = d->nx, ny = d->ny, nz = d->nz;
    if ((long long)nx * ny * nz > kNaMaxCells || nx > kNaMaxN || ny > kNaMaxN || nz > kNaMaxNz)
        return FIZZY_ERR_UNSUPPORTED;
    // set-up, once per device, with that device current
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return FIZZY_ERR_CUDA;
    if (!g_noalloc_dev[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            (void)cudaGetLastError();
            return FIZZY_ERR_CUDA;
        }
        g_noalloc_dev[dev] = (double *)ptr;
    }
    double *S = g_noalloc_dev[dev];
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)nx * ny * nz;

    // ---- device regions
    double *qx = S, *qy = S + kNaMaxCells, *qz = S + 2 * (size_t)kNaMaxCells;
    double *fhat = S + 3 * (size_t)kNaMaxCells;
    double *dtab = S + 4 * (size_t)kNaMaxCells;  // m | ib | z tables | cup | fft tables
    // ---- host tables, laid out exactly like the device region starting at dtab
    double *H = g_noalloc_host;
    const int Ux = d->bc_x == FIZZY_BC_PERIODIC ? nx / 2 + 1 : nx;
    const int Uy = d->bc_y == FIZZY_BC_PERIODIC ? ny / 2 + 1 : ny;
    const size_t ts = (size_t)Ux * Uy;
    double *hm = H, *hib = H + kNaMaxCells;
    double *hz = H + 2 * (size_t)kNaMaxCells;       // kNaZTabs x kNaMaxNz
    double *hcup = hz + kNaZTabs * (size_t)kNaMaxNz;
    double *hfft = hcup + kNaMaxNz;                 // tw_x | cs_x | tw_y | cs_y
    static double zf[kNaMaxNz + 1], zc[kNaMaxNz];
    for (int k = 0; k <= nz; ++k) zf[k] = d->zf ? d->zf[k] : d->dz * k;
    for (int k = 0; k < nz; ++k) zc[k] = 0.5 * (zf[k] + zf[k + 1]);
    double lz = 0.0;
    const double sig = 1.0 / (4.0 * (double)nx * (double)ny);
    // per-k tables (same definitions and arithmetic as the plan's)
    enum { Z_FAZ, Z_FRZ, Z_DVZ, Z_DVZS, Z_CGZ, Z_LZA, Z_LZC, Z_IZF, Z_DZF, Z_DZC };
    static_assert(Z_LZA == kZPhys && Z_DZC + 1 == kNaZTabs, "per-k table layout");
    for (int k = 0; k < nz; ++k) lz += zf[k + 1] - zf[k];
    for (int k = 0; k < nz; ++k) {
        const double dzf_k = zf[k + 1] - zf[k];
        const bool top = (k == nz - 1);
        const double dzc_k = top ? 0.0 : zc[k + 1] - zc[k];
        const double dzc_km = (k > 0) ? zc[k] - zc[k - 1] : 0.0;
        physics_zrow(d->rho_l, d->rho_g, d->dt, sig, dzf_k, dzc_k, top, &hz[k], kNaMaxNz);
        hz[Z_LZA * kNaMaxNz + k] = (k > 0) ? 1.0 / (dzf_k * dzc_km) : 0.0;
        hz[Z_LZC * kNaMaxNz + k] = top ? 0.0 : 1.0 / (dzf_k * dzc_k);
        hz[Z_IZF * kNaMaxNz + k] = 1.0 / dzf_k;
        hz[Z_DZF * kNaMaxNz + k] = dzf_k;
        hz[Z_DZC * kNaMaxNz + k] = dzc_k;
        hcup[k] = hz[Z_LZC * kNaMaxNz + k];
    }
    // transform tables
    fill_fft_tables(nx, hfft, hfft + kNaTw);
    fill_fft_tables(ny, hfft + kNaTw + kNaCs, hfft + 2 * kNaTw + kNaCs);
    // z factorisation per distinct eigenvalue pair
    const double *A = &hz[Z_LZA * kNaMaxNz];
    const double *C = &hz[Z_LZC * kNaMaxNz];
    for (size_t uu = 0; uu < ts; ++uu) {
        const int ux = (int)(uu % Ux), uy = (int)(uu / Ux);
        if (ux == 0 && uy == 0) {
            for (int k = 0; k < nz; ++k) hm[(size_t)k * ts] = hib[(size_t)k * ts] = 0.0;
            continue;
        }
        const double lam = eig(ux, nx, d->dx, d->bc_x) + eig(uy, ny, d->dy, d->bc_y);
        double beta = -(A[0] + C[0]) + lam;
        hm[uu] = 0.0;
        hib[uu] = 1.0 / beta;
        for (int k = 1; k < nz; ++k) {
            const double m = A[k] / beta;
            beta = (-(A[k] + C[k]) + lam) - m * C[k - 1];
            hm[(size_t)k * ts + uu] = m;
            hib[(size_t)k * ts + uu] = 1.0 / beta;
        }
    }
    // copy the used parts: m and 1/beta tables, then per-k + transform tables
    cudaError_t e = cudaMemcpyAsync(dtab, hm, ts * nz * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtab + kNaMaxCells, hib, ts * nz * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtab + 2 * (size_t)kNaMaxCells, hz,
                            ((kNaZTabs + 1) * (size_t)kNaMaxNz + 2 * (kNaTw + kNaCs)) * sizeof(double),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return FIZZY_ERR_CUDA;
    }

    // ---- kernel arguments pointing into the scratch
    double *dz_ = dtab + 2 * (size_t)kNaMaxCells;
    double *dcup = dz_ + kNaZTabs * (size_t)kNaMaxNz;
    double *dfft = dcup + kNaMaxNz;
    GridDev g;
    memset(&g, 0, sizeof(g));
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.bcx = d->bc_x;
    g.bcy = d->bc_y;
    g.perz = d->periodic_z ? 1 : 0;
    g.sing = (d->bc_x <= FIZZY_BC_NEUMANN && d->bc_y <= FIZZY_BC_NEUMANN) ? 1 : 0;
    g.rny = (unsigned)((1ull << 32) / (unsigned)ny + 1);
    physics_consts(g, d->rho_l, d->rho_g, d->dt, d->dx, d->dy, sig);
    g.idx2 = 1.0 / (d->dx * d->dx);
    g.idy2 = 1.0 / (d->dy * d->dy);
    g.idx1 = 1.0 / d->dx;
    g.idy1 = 1.0 / d->dy;
    g.faz = dz_ + Z_FAZ * kNaMaxNz;
    g.frz = dz_ + Z_FRZ * kNaMaxNz;
    g.dvz = dz_ + Z_DVZ * kNaMaxNz;
    g.dvz_s = dz_ + Z_DVZS * kNaMaxNz;
    g.cgz = dz_ + Z_CGZ * kNaMaxNz;
    g.lza = dz_ + Z_LZA * kNaMaxNz;
    g.lzc = dz_ + Z_LZC * kNaMaxNz;
    g.izf = dz_ + Z_IZF * kNaMaxNz;
    g.dzf = dz_ + Z_DZF * kNaMaxNz;
    g.dzc = dz_ + Z_DZC * kNaMaxNz;
    g.inv_lz = 1.0 / lz;
    g.sigma = sig;
    g.div_tol = -1.0;
    FFTDesc Dx, Dy;
    memset(&Dx, 0, sizeof(Dx));
    memset(&Dy, 0, sizeof(Dy));
    fill_stages(Dx, nx);
    Dx.kind = d->bc_x == FIZZY_BC_NEUMANN ? KIND_DCT : KIND_PERIODIC;
    Dx.tw = dfft;
    Dx.cs = dfft + kNaTw;
    fill_stages(Dy, ny);
    Dy.kind = d->bc_y == FIZZY_BC_NEUMANN ? KIND_DCT : KIND_PERIODIC;
    Dy.tw = dfft + kNaTw + kNaCs;
    Dy.cs = dfft + 2 * kNaTw + kNaCs;
    const int Lx = x_lines_per_cta(nx), TXy = y_tile_cols(ny);
    const size_t smx = pass_smem<double>(nx, Lx), smy = pass_smem<double>(ny, TXy / 2);
    const dim3 cblk(32, 8), cgrd((nx + 31) / 32, (ny + 7) / 8, nz);
    const int xtiles = (ny * nz + 2 * Lx - 1) / (2 * Lx);
    const int ygx = (nx + TXy - 1) / TXy, ytiles = ygx * nz;
    const int ttiles = (nx * ny + THOMAS_BLOCK - 1) / THOMAS_BLOCK;  // one z-line per thread
    auto grid = [&](int tiles, int) { return std::max(1, tiles); };  // one block per tile
    XArgs xa;
    memset(&xa, 0, sizeof(xa));
    xa.qx = qx;
    xa.qy = qy;
    xa.qz = qz;
    xa.out = fhat;
    (void)N;

    const dim3 fgrd = flux_grid(nx, ny, nz), fblk(FLUX_BX, FLUX_BY);
    if (d->rho_g <= d->rho_l)
        k_flux<true><<<fgrd, fblk, 0, s>>>(g, kFluxKc, phi, p_n, p_nm1, u, v, w, qx, qy, qz, nullptr);
    else
        k_flux<false><<<fgrd, fblk, 0, s>>>(g, kFluxKc, phi, p_n, p_nm1, u, v, w, qx, qy, qz, nullptr);
    k_xfwd<double, XF_F64_DIVQ><<<grid(xtiles, CAP_XF64), 256, smx, s>>>(g, Dx, Lx, xa, xtiles);
    k_ypass<double, false><<<grid(ytiles, CAP_Y64F), 256, smy, s>>>(nx, ny, Dy, TXy, fhat, nullptr, ygx, ytiles);
    k_thomas<double><<<grid(ttiles, CAP_TH64), THOMAS_BLOCK, thomas_smem<double>(), s>>>(g, Ux, Uy, dtab, dtab + kNaMaxCells, dcup, fhat, nullptr, ttiles);
    k_ypass<double, true><<<grid(ytiles, CAP_Y64I), 256, smy, s>>>(nx, ny, Dy, TXy, fhat, nullptr, ygx, ytiles);
    k_xinv<double, XI_STORE><<<grid(xtiles, CAP_XI64), 256, smx, s>>>(g, Dx, Lx, fhat, p_np1, nullptr, xtiles);
    k_correct<<<cgrd, cblk, 0, s>>>(g, p_np1, qx, qy, qz, u, v, w);
    e = cudaGetLastError();
    return e == cudaSuccess ? FIZZY_OK : FIZZY_ERR_CUDA;
}
