// Real-to-real transforms along x and y for the fast Poisson solver
// (CaNS-style direct solver, paper "Methods and Implementation strategy":
// FFT along the periodic directions; here also the DCT-II basis for walls).
//
// Scheme (own design for sm_103a):
//  * Two real lines a, b are packed into one complex line z = a + i b and
//    transformed by a single complex FFT; the two real spectra are separated
//    afterwards with Z[m] and conj(Z[n-m]).
//  * Periodic direction: real DFT in half-complex order (index m <= n/2 holds
//    Re A_m, index n-m holds Im A_m).  Wall direction: DCT-II obtained from the
//    same FFT after the even/odd reordering of Makhoul (1980),
//    v_t = x_2t, v_(n-1-t) = x_(2t+1), and a post-twiddle exp(-i pi m / (2n)).
//  * Both forward variants output 2x the plain sums and both inverse variants
//    return 2n x the input, so a 2-D round trip scales by 4 nx ny; the solver
//    folds 1/(4 nx ny) into the right-hand side.
//  * The complex FFT is a Stockham autosort (self-sorting) mixed-radix
//    (4, 2, 3) FFT in shared memory with ping-pong buffers and one barrier per
//    stage; twiddles come from a per-plan table staged into shared memory,
//    in the FMA-friendly form described at tw_apply.
#pragma once
#include "kern_common.cuh"

namespace fz {

// Transform kinds.  KIND_DCT4 (zero flux at the near face, p = 0 at the far
// face) is the DCT-IV, X_k = sum_n x_n cos(pi (2n+1)(2k+1) / (4n)), computed
// per real line by one complex FFT of half the length (see dct4_tile).  The
// descriptor's flip turns a DCT-II into the DST-II (p = 0 at both faces) and
// a DCT-IV into the DST-IV (p = 0 near, zero flux far): with y_n = (-1)^n x_n,
//     DST-II(x)_k = DCT-II(y)_(N-1-k),   DST-IV(x)_k = DCT-IV(y)_(N-1-k),
// so the forward pass negates the odd samples on loading and the inverse
// pass negates them on storing; the reversed spectral index is absorbed into
// the eigenvalue of each slot (slot j holds the sine index N-1-j).
enum { KIND_PERIODIC = 0, KIND_DCT = 1, KIND_DCT4 = 2 };

constexpr int FFT_MAX_STAGES = 12;

// One transform direction (kernel argument, by value).  Per stage s: radix
// rad[s], butterfly stride m[s] = n/rad[s], span ns[s] (product of the
// earlier radices), twiddle step twq[s] = n/(ns[s] rad[s]) and the
// multiply-high reciprocals of m[s] and ns[s]: for 0 <= x < 2^31/d,
// floor(x/d) = umulhi(x, floor(2^32/d) + 1)  (d > 1).
struct FFTDesc {
    int n;           // line length (the complex FFT length too, except KIND_DCT4: n/2)
    int nst;         // number of Stockham stages
    int kind;        // KIND_PERIODIC, KIND_DCT or KIND_DCT4
    int flip;        // 1: negate odd samples (DST-II from KIND_DCT, DST-IV from KIND_DCT4)
    unsigned rK;     // KIND_DCT4: multiply-high reciprocal of n/2
    int rad[FFT_MAX_STAGES], m[FFT_MAX_STAGES], ns[FFT_MAX_STAGES], twq[FFT_MAX_STAGES];
    unsigned rm[FFT_MAX_STAGES], rns[FFT_MAX_STAGES];
    unsigned rn, rM;  // multiply-high reciprocals of n and M = n/2 + 1
    const void *tw;  // n entries (m, tau) of exp(-2 pi i t / n), see tw_apply (T2); KIND_DCT4:
                     // n/2 such entries for length n/2, then the pre-twiddles
                     // exp(-i pi (4t+1)/(4n)), t < n/2
    const void *cs;  // n/2+1 complex: (cos, sin)(pi m / (2 n)) (T2); KIND_DCT4: the
                     // post-twiddles 2 exp(-i pi k / n), k < n/2
};

__device__ __forceinline__ int fdiv(int x, int d, unsigned r) {
    return d == 1 ? x : (int)__umulhi((unsigned)x, r);
}
// The multiply-high reciprocal of d, for fdiv (exact for 0 <= x < 2^32/d).
__device__ __forceinline__ unsigned fdiv_recip(int d) {
    return d > 1 ? 0xffffffffu / (unsigned)d + 1u : 0u;
}

// position of input sample i inside the (possibly reordered) complex line
__device__ __forceinline__ int line_pos(int i, int n, int kind) {
    return (kind == KIND_DCT) ? ((i & 1) ? n - 1 - (i >> 1) : (i >> 1)) : i;
}

// Twiddle factors are stored in an FMA-friendly form: for w = c + i s the
// table entry is (m, tau) with
//     w = m (1 + i tau)       (R = 0, |c| >= |s|: m = c, tau = s/c)
//     w = i m (1 + i tau)     (R = 1, |c| <  |s|: m = s, tau = -c/s)
// so |tau| <= 1, and R is kept in the lowest mantissa bit of tau (a
// perturbation of at most one unit in the last place).  Multiplying x by w
// (or by conj(w) for the inverse) is then z = x (1 +- i tau) (2 FMAs)
// followed by a scale by m that folds into the FMAs of the butterfly: the
// product is (mr * za, mi * zb) with (za, zb) = (z.re, z.im) or (z.im, z.re)
// and (mr, mi) = (+-m, +-m).  A radix-4 butterfly with its three twiddles
// (w3 = w1 w2: c = w1 (x1 + w2 x3), d = w1 (x1 - w2 x3)) costs 24 FMAs
// instead of 12 multiply-adds for the twiddles and 16 adds; radix 2 costs 6
// instead of 8.
template <typename T> struct TwApplied {
    T za, zb, mr, mi;  // w x = (mr za, mi zb)
};

__device__ __forceinline__ bool tw_rot(double tau) { return __double2loint(tau) & 1; }
__device__ __forceinline__ bool tw_rot(float tau) { return __float_as_uint(tau) & 1u; }
__device__ __forceinline__ double flip_sign(double v, bool f) {
    return __hiloint2double(__double2hiint(v) ^ (f ? (int)0x80000000 : 0), __double2loint(v));
}
__device__ __forceinline__ float flip_sign(float v, bool f) {
    return __uint_as_float(__float_as_uint(v) ^ (f ? 0x80000000u : 0u));
}

// x times w (INV: times conj(w)); w = (m, tau) from the table.
template <typename T, bool INV>
__device__ __forceinline__ TwApplied<T> tw_apply(typename C2<T>::t x, typename C2<T>::t w) {
    const T m = w.x, tau = w.y;
    const bool R = tw_rot(tau);
    T zr, zi;
    if (!INV) {  // x (1 + i tau)
        zr = fmaT(-tau, x.y, x.x);
        zi = fmaT(tau, x.x, x.y);
    } else {     // x (1 - i tau)
        zr = fmaT(tau, x.y, x.x);
        zi = fmaT(-tau, x.x, x.y);
    }
    TwApplied<T> o;
    o.za = R ? zi : zr;
    o.zb = R ? zr : zi;
    // R = 1: i m z = (-m zi, m zr); inverse: -i m z = (m zi, -m zr)
    o.mr = flip_sign(m, R && !INV);
    o.mi = flip_sign(m, R && INV);
    return o;
}

// One Stockham stage over L lines (line stride ls) from src to dst.  FIXED:
// the stage constants are compile-time values (a length-specialised
// transform), so the divisions are written out and fold to shifts.
template <typename T, bool INV, bool FIXED = false>
__device__ __forceinline__ void stockham_stage(const typename C2<T>::t *__restrict__ src,
                                               typename C2<T>::t *__restrict__ dst, int L, int ls,
                                               int R, int m, unsigned rm, int Ns, unsigned rns,
                                               int twq, const typename C2<T>::t *__restrict__ tw) {
    typedef typename C2<T>::t T2;
    const int total = L * m;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int l = FIXED ? t / m : fdiv(t, m, rm);
        const int b = t - l * m;
        const int j = FIXED ? b % Ns : b - fdiv(b, Ns, rns) * Ns;
        const T2 *in = src + l * ls + b;
        T2 *out = dst + l * ls + (b - j) * R + j;
        const int ts = j * twq;
        if (R == 4) {
            const T2 x0 = in[0], x1 = in[m], x2 = in[2 * m], x3 = in[3 * m];
            if (Ns == 1) {  // no twiddles
                const T ar = x0.x + x2.x, ai = x0.y + x2.y;
                const T br = x0.x - x2.x, bi = x0.y - x2.y;
                const T cr = x1.x + x3.x, ci = x1.y + x3.y;
                const T dr = x1.x - x3.x, di = x1.y - x3.y;
                out[0] = mk2(ar + cr, ai + ci);
                out[2 * Ns] = mk2(ar - cr, ai - ci);
                if (!INV) {  // y1 = b - i d, y3 = b + i d
                    out[Ns] = mk2(br + di, bi - dr);
                    out[3 * Ns] = mk2(br - di, bi + dr);
                } else {     // y1 = b + i d, y3 = b - i d
                    out[Ns] = mk2(br - di, bi + dr);
                    out[3 * Ns] = mk2(br + di, bi - dr);
                }
            } else {
                const T2 w1 = tw[ts], w2 = tw[2 * ts];
                // a, b = x0 +- w2 x2;  e, f = x1 +- w2 x3
                const TwApplied<T> X2 = tw_apply<T, INV>(x2, w2);
                const T ar = fmaT(X2.mr, X2.za, x0.x), ai = fmaT(X2.mi, X2.zb, x0.y);
                const T br = fmaT(-X2.mr, X2.za, x0.x), bi = fmaT(-X2.mi, X2.zb, x0.y);
                const TwApplied<T> X3 = tw_apply<T, INV>(x3, w2);
                T2 e, f;
                e.x = fmaT(X3.mr, X3.za, x1.x);
                e.y = fmaT(X3.mi, X3.zb, x1.y);
                f.x = fmaT(-X3.mr, X3.za, x1.x);
                f.y = fmaT(-X3.mi, X3.zb, x1.y);
                // c = w1 e, d = w1 f;  y0, y2 = a +- c
                const TwApplied<T> C = tw_apply<T, INV>(e, w1);
                out[0] = mk2(fmaT(C.mr, C.za, ar), fmaT(C.mi, C.zb, ai));
                out[2 * Ns] = mk2(fmaT(-C.mr, C.za, ar), fmaT(-C.mi, C.zb, ai));
                const TwApplied<T> D = tw_apply<T, INV>(f, w1);  // d = (D.mr D.za, D.mi D.zb)
                if (!INV) {  // y1 = b - i d, y3 = b + i d
                    out[Ns] = mk2(fmaT(D.mi, D.zb, br), fmaT(-D.mr, D.za, bi));
                    out[3 * Ns] = mk2(fmaT(-D.mi, D.zb, br), fmaT(D.mr, D.za, bi));
                } else {     // y1 = b + i d, y3 = b - i d
                    out[Ns] = mk2(fmaT(-D.mi, D.zb, br), fmaT(D.mr, D.za, bi));
                    out[3 * Ns] = mk2(fmaT(D.mi, D.zb, br), fmaT(-D.mr, D.za, bi));
                }
            }
        } else if (R == 2) {
            const T2 x0 = in[0], x1 = in[m];
            if (Ns == 1) {
                out[0] = mk2(x0.x + x1.x, x0.y + x1.y);
                out[Ns] = mk2(x0.x - x1.x, x0.y - x1.y);
            } else {
                const TwApplied<T> X1 = tw_apply<T, INV>(x1, tw[ts]);
                out[0] = mk2(fmaT(X1.mr, X1.za, x0.x), fmaT(X1.mi, X1.zb, x0.y));
                out[Ns] = mk2(fmaT(-X1.mr, X1.za, x0.x), fmaT(-X1.mi, X1.zb, x0.y));
            }
        } else {  // R == 3
            T2 x0 = in[0], x1 = in[m], x2 = in[2 * m];
            if (Ns > 1) {
                const TwApplied<T> X1 = tw_apply<T, INV>(x1, tw[ts]);
                const TwApplied<T> X2 = tw_apply<T, INV>(x2, tw[2 * ts]);
                x1 = mk2(mulT(X1.mr, X1.za), mulT(X1.mi, X1.zb));
                x2 = mk2(mulT(X2.mr, X2.za), mulT(X2.mi, X2.zb));
            }
            const T h = (T)0.86602540378443864676;  // sqrt(3)/2
            const T sr = x1.x + x2.x, si = x1.y + x2.y;
            const T mr = fmaT((T)-0.5, sr, x0.x), mi = fmaT((T)-0.5, si, x0.y);
            const T dx = x1.x - x2.x, dy = x1.y - x2.y;
            out[0] = mk2(x0.x + sr, x0.y + si);
            if (!INV) {  // y1 = m - i h d, y2 = m + i h d
                out[Ns] = mk2(fmaT(h, dy, mr), fmaT(-h, dx, mi));
                out[2 * Ns] = mk2(fmaT(-h, dy, mr), fmaT(h, dx, mi));
            } else {
                out[Ns] = mk2(fmaT(-h, dy, mr), fmaT(h, dx, mi));
                out[2 * Ns] = mk2(fmaT(h, dy, mr), fmaT(-h, dx, mi));
            }
        }
    }
}

// Full complex FFT of L lines; data starts in a, b is the other buffer.
// Returns the buffer that holds the result.  Ends with a barrier.
template <typename T, bool INV>
__device__ typename C2<T>::t *fft_lines(typename C2<T>::t *a, typename C2<T>::t *b, int L, int ls,
                                        const FFTDesc &D, const typename C2<T>::t *tw) {
#pragma unroll
    for (int s = 0; s < FFT_MAX_STAGES; ++s) {
        if (s >= D.nst) break;
        stockham_stage<T, INV>(a, b, L, ls, D.rad[s], D.m[s], D.rm[s], D.ns[s], D.rns[s], D.twq[s], tw);
        __syncthreads();
        typename C2<T>::t *t = a;
        a = b;
        b = t;
    }
    return a;
}

// Radix plan of a compile-time length (radix 4 first, then 2, then 3, the
// order the host uses): number of stages and the constants of stage s.
constexpr int plan_radix(int n, int s) {
    for (int k = 0;; ++k) {
        const int r = (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : 1;
        if (r == 1) return 1;
        if (k == s) return r;
        n /= r;
    }
}
constexpr int plan_nst(int n) {
    int s = 0;
    while (plan_radix(n, s) != 1) ++s;
    return s;
}
constexpr int plan_span(int n, int s) {  // product of the radices before stage s
    int ns = 1;
    for (int k = 0; k < s; ++k) ns *= plan_radix(n, k);
    return ns;
}

// Full complex FFT of L lines of compile-time length N (stages unrolled with
// constant R, m, Ns and twiddle step); same result as fft_lines.
template <typename T, bool INV, int N, int S = 0>
__device__ __forceinline__ typename C2<T>::t *fft_fixed(typename C2<T>::t *a, typename C2<T>::t *b,
                                                        int L, int ls, const typename C2<T>::t *tw) {
    if constexpr (S >= plan_nst(N)) {
        return a;
    } else {
        constexpr int R = plan_radix(N, S), NS = plan_span(N, S);
        stockham_stage<T, INV, true>(a, b, L, ls, R, N / R, 0u, NS, 0u, N / (NS * R), tw);
        __syncthreads();
        return fft_fixed<T, INV, N, S + 1>(b, a, L, ls, tw);
    }
}

// Stage the twiddle tables of D into shared memory (tw: n entries, cs: n/2+1).
template <typename T>
__device__ __forceinline__ void load_tables(const FFTDesc &D, typename C2<T>::t *tw_s,
                                            typename C2<T>::t *cs_s) {
    typedef typename C2<T>::t T2;
    const T2 *tw = (const T2 *)D.tw;
    const T2 *cs = (const T2 *)D.cs;
    for (int t = threadIdx.x; t < D.n; t += blockDim.x) tw_s[t] = tw[t];
    if (D.kind == KIND_DCT)
        for (int t = threadIdx.x; t <= D.n / 2; t += blockDim.x) cs_s[t] = cs[t];
    if (D.kind == KIND_DCT4)
        for (int t = threadIdx.x; t < D.n / 2; t += blockDim.x) cs_s[t] = cs[t];
}

// a sample of a flipped direction: odd samples negated (an integer operation)
template <typename T> __device__ __forceinline__ T flip_odd(T v, int flip, int i) {
    return flip_sign(v, flip && (i & 1));
}

// Forward separation for the pair index m of one complex line Z (length n):
// writes the two real spectra (scaled by 2) through out(a_or_b, index, value).
template <typename T, typename F>
__device__ __forceinline__ void fwd_separate(const typename C2<T>::t *Z, int n, int m, int kind,
                                             const typename C2<T>::t *cs, F &&out) {
    typedef typename C2<T>::t T2;
    if (m == 0) {
        const T2 z = Z[0];
        out(0, 0, z.x + z.x);
        out(1, 0, z.y + z.y);
        return;
    }
    const T2 z = Z[m];
    if (2 * m == n) {  // Nyquist (even n): both spectra are real there
        const T f = (kind == KIND_DCT) ? (T)1.41421356237309504880 : (T)2;  // 2 cos(pi/4) or 2
        out(0, m, f * z.x);
        out(1, m, f * z.y);
        return;
    }
    const T2 y = Z[n - m];
    const T var = z.x + y.x, vai = z.y - y.y;  // 2 A_m
    const T vbr = z.y + y.y, vbi = y.x - z.x;  // 2 B_m
    if (kind == KIND_PERIODIC) {
        out(0, m, var);
        out(0, n - m, vai);
        out(1, m, vbr);
        out(1, n - m, vbi);
    } else {  // X[m] = Re(w V), X[n-m] = -Im(w V), w = c - i s
        const T c = cs[m].x, s = cs[m].y;
        out(0, m, fmaT(c, var, mulT(s, vai)));
        out(0, n - m, fmaT(s, var, -mulT(c, vai)));
        out(1, m, fmaT(c, vbr, mulT(s, vbi)));
        out(1, n - m, fmaT(s, vbr, -mulT(c, vbi)));
    }
}

// Inverse combination for pair index m: given the real spectra values of lines
// a and b (get(a_or_b, index)), writes Z[m] and Z[n-m] of the packed line.
template <typename T, typename G>
__device__ __forceinline__ void inv_combine(typename C2<T>::t *Z, int n, int m, int kind,
                                            const typename C2<T>::t *cs, G &&get) {
    if (m == 0) {
        Z[0] = mk2(get(0, 0), get(1, 0));
        return;
    }
    if (2 * m == n) {
        const T f = (kind == KIND_DCT) ? (T)1.41421356237309504880 : (T)1;
        Z[m] = mk2(f * get(0, m), f * get(1, m));
        return;
    }
    T ar, ai, br, bi;
    if (kind == KIND_PERIODIC) {
        ar = get(0, m);
        ai = get(0, n - m);
        br = get(1, m);
        bi = get(1, n - m);
    } else {  // V[m] = (c + i s)(X[m] - i X[n-m])
        const T c = cs[m].x, s = cs[m].y;
        const T xa = get(0, m), ya = get(0, n - m), xb = get(1, m), yb = get(1, n - m);
        ar = fmaT(c, xa, mulT(s, ya));
        ai = fmaT(s, xa, -mulT(c, ya));
        br = fmaT(c, xb, mulT(s, yb));
        bi = fmaT(s, xb, -mulT(c, yb));
    }
    Z[m] = mk2(ar - bi, ai + br);
    Z[n - m] = mk2(ar + bi, br - ai);
}

}  // namespace fz
