/*
 * lbve_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * Plain, slow FP64 CPU oracle of the hybrid lattice-Boltzmann scheme for the integral nonlinear
 * Maxwell (nlM) fluid of Papenkort & Voigtmann, "Lattice Boltzmann simulations of a viscoelastic
 * shear-thinning fluid" (arXiv:1504.06123).  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code, header, table or
 * constant with the CUDA library: every lattice table and formula below is written out here again.
 *
 * Storage follows the paper's own scheme (Sec. III, Eq. (eeval)): every history point keeps the
 * velocity gradient kappa it was created with and its factor exp(kappa dt_b); the deformation
 * tensor E(t,t') is re-formed every step as the ordered product of the stored factors, newest on
 * the left.  (The CUDA path instead updates E - I in place, so the two are independent
 * algorithms.)
 *
 * Conventions
 *   Populations are kept as deviations dn_i = n_i - w_i rho0 from the rest state.  This is an exact
 *   re-parametrisation of the collide-stream rule (both are linear in n), chosen so that FP64 resolves
 *   velocities of 1e-6 to 1e-16 relative instead of to the ~1e-10 left by rounding populations of 0.4.
 *   kappa[a][b] = d v_a / d x_b  (kappa = (grad v)^T, Sec. I), stored row-major, d*d entries.
 *   sigma components: 2D xx, yy, xy; 3D xx, yy, zz, xy, xz, yz.
 *   Node index: x fastest, then y, then z.  Node j of a walled axis sits at j, walls at -1/2 and
 *   n-1/2 (half-way bounce-back).
 *   Lattice units dt = dx = 1.
 *
 * Pins (tests/test_oracle_*.py check this file against the paper and the mathematics, not against itself):
 * exp of the factors vs scipy's expm; the history grid vs an independent enumeration; E(t,t) = 1; constant
 * simple shear in closed form; the Maxwell / nlM continuum limit; brute force from raw per-step factor
 * products on tiny grids; Newtonian Poiseuille with the BGK bounce-back slip and its Fourier startup
 * series; the UCM steady parabola; the nlM force balance; mass conservation of the density source;
 * x-invariance and channel / duct symmetries; post-collision moments of Eq. (bodyforce); Eq. (inlM) vs the
 * nilpotent closed form, the extensional geometric series, the steady UCM solve and the Laplace integral;
 * White-Metzner vs brute-force strain sums; the pressure-step boundary vs the BGK Poiseuille solution and
 * the equivalent body force; the startup / cessation features Sec. IV states (overshoot, counter-flow,
 * sign and decay of the normal-stress difference, Newtonian / UCM symmetry).
 * Parity unpinned beyond the stated readings: the kappa averaging of a merge (pinned only by the
 * brute-force check of the merge rule), the choice of trace terms with trace_full = 0 (pinned only through
 * mass conservation), and the wall-adjacent finite-difference stencil (exact on parabolas; the steady
 * channels pin it only to 1e-3).
 *
 * Readings of the paper taken here (the same readings are used by the CUDA path):
 *   - factor for the interval [t, t+1] is exp(kappa(t)) (explicit, Eq. (eeval));
 *   - the new point of step t sits at age 0 with E = 1 and kappa(t);
 *   - history blocks start full of rest points (E = 1, kappa = 0) on the quasi-log grid; inserting
 *     into a full block b > 1 first moves its two oldest points, merged, into block b-1 (older
 *     point's time and E, averaged kappa, factor = product); a full block 1 drops its oldest point
 *     (Sec. III, quasi-logarithmic memory layout);
 *   - second exponential of Eq. (nlmax) uses (t - t') |gammadot(t')| (no measure "dt'");
 *   - gammadot^2 = (1/2) tr D^2, D = kappa + kappa^T (Sec. II);
 *   - trapezoidal rule on the non-uniform age grid of the retained points (Sec. III);
 *   - -d_{t'} B = E kappa(t') E^T + (E kappa(t') E^T)^T (Sec. III; the text writes d_t);
 *   - density source d_t(delta rho) = -(tr sigma(t) - tr sigma(t-1)) / (d c_s^2) and the hydrodynamic
 *     density rho = sum n + (1/2) d_t(delta rho), momentum rho u = sum c n + f/2 (Eq. (hydrofields));
 *     kappa(t) is taken from the raw velocity (sum c n + f/2) / sum n because the corrected density
 *     needs sigma(t) itself;
 *   - forcing term F_i exactly as Eq. (bodyforce) with f = rho0 g; trace_full = 0 drops both
 *     d_t(delta rho) terms and uses rho = sum n (the "standard" fields of the channel simplification);
 *   - the Newtonian background viscosity of Eq. (nlM) is the BGK viscosity rho c_s^2 (tau_LB - 1/2);
 *   - kappa by second-order finite differences: central in the bulk and on periodic axes; at a
 *     wall-adjacent node the three-point formula through the no-slip wall half a node away.
 *
 * Constitutive variants of sigma_struc (model kind, Sec. II and Sec. IV):
 *   - ORC_NLM: the integral nlM, Eq. (gitt) with the modulus of Eq. (nlmax) (default);
 *   - ORC_INLM: the instantaneous nlM, Eq. (inlM) re-read as a stress / strain-rate law at time t:
 *     sigma_struc(t) = G_inf sum_{n>=1} tau_M^n d^(n)[kappa(t)], tau_M = (1/tau + gammadot(t)/gamma_c)^-1
 *     (the steady form of Eq. (nlmax)), the series summed term by term until it has converged; where
 *     it does not converge (no steady state exists) the stress is NaN;
 *   - ORC_WM: the White-Metzner form of Eq. (nlmax): the second exponential uses the strain
 *     accumulated between t' and t, sum_{s=t'}^{t-1} gammadot(s) (the same explicit left-end rule as
 *     the factors of Eq. (eeval)), instead of (t - t') gammadot(t').  Every point stores the strain of
 *     its span next to its factor; a merge adds the two spans' strains, as it multiplies their factors.
 *
 * Threads: the node loops (moments, gradient, history, collision and streaming, the history-only driver)
 * may run on several host threads (OpenMP, orc_set_threads).  Each node's arithmetic is the same
 * sequence of operations whatever the thread count -- threads only split the nodes, and every node's
 * result is written by exactly one thread -- so results are bitwise independent of the thread count.
 *
 * Pressure-step boundary along x (Sec. III, the generalised periodic boundary of Kim & Pitsch that fixes a
 * constant pressure step between the inlet and the outlet of the periodic lattice), optional: the
 * periodic images just outside the lattice are ghost nodes.  The ghost upstream of the inlet (x = -1)
 * carries the outlet node's (x = nx-1) post-collision non-equilibrium populations on an equilibrium at the
 * inlet density rho_in and the outlet node's velocity; the ghost downstream of the outlet (x = nx) carries
 * the inlet node's non-equilibrium populations on an equilibrium at rho_out and the inlet node's velocity.
 * Populations crossing the seam stream from these ghosts: n_ghost = n_eq(rho_ghost, u) + (n* - n_eq(rho, u)),
 * rho and u the hydrodynamic fields of the node whose populations are imaged.  dp is the pressure drop over
 * one period (nx spacings); the ghosts sit on that linear profile, nx + 1 spacings apart around the mean
 * rho0: rho_in/out = rho0 +- (dp / c_s^2) (nx + 1) / (2 nx).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads of the node loops (1 = serial). */
static int orc_nthreads = 1;

/* Set the number of host threads of the node loops (n < 1: all available); returns the number in use
 * (1 when the library was built without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    orc_nthreads = (n < 1) ? omp_get_num_procs() : n;
#else
    (void)n;
    orc_nthreads = 1;
#endif
    return orc_nthreads;
}

int orc_get_threads(void) { return orc_nthreads; }

#define ORC_MAXQ 19

/* ------------------------------------------------------------------------------------------ */
/* Small dense matrix helpers (d = 2 or 3, row-major).                                          */
/* ------------------------------------------------------------------------------------------ */

static void mat_identity(int d, double* A) {
    for (int i = 0; i < d * d; ++i) A[i] = 0.0;
    for (int i = 0; i < d; ++i) A[i * d + i] = 1.0;
}

/* C = A * B  (C may not alias A or B) */
static void mat_mul(int d, const double* A, const double* B, double* C) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += A[i * d + k] * B[k * d + j];
            C[i * d + j] = s;
        }
}

/* C = A * B^T */
static void mat_mul_bt(int d, const double* A, const double* B, double* C) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += A[i * d + k] * B[j * d + k];
            C[i * d + j] = s;
        }
}

/*
 * Matrix exponential of a 2x2 matrix, closed form.  With m = tr K / 2 and K0 = K - m I (traceless),
 * K0^2 = q I where q = ((a-d)/2)^2 + b c = -det K0, hence
 *     exp(K) = e^m ( ch(q) I + sh(q) K0 ),  ch(q) = cosh(sqrt q), sh(q) = sinh(sqrt q)/sqrt q,
 * both entire functions of q (cos/sin for q < 0).  Small |q| uses their power series.
 */
static void expm2(const double* K, double* out) {
    const double a = K[0], b = K[1], c = K[2], d = K[3];
    const double m = 0.5 * (a + d);
    const double h = 0.5 * (a - d);
    const double q = h * h + b * c;
    double ch, sh;
    if (fabs(q) < 1e-6) {
        /* sum_n q^n/(2n)! and sum_n q^n/(2n+1)!, converged to below 1e-32 */
        double tc = 1.0, ts = 1.0;
        ch = 1.0;
        sh = 1.0;
        for (int n = 1; n < 12; ++n) {
            tc *= q / ((2.0 * n - 1.0) * (2.0 * n));
            ts *= q / ((2.0 * n) * (2.0 * n + 1.0));
            ch += tc;
            sh += ts;
        }
    } else if (q > 0) {
        const double r = sqrt(q);
        ch = cosh(r);
        sh = sinh(r) / r;
    } else {
        const double r = sqrt(-q);
        ch = cos(r);
        sh = sin(r) / r;
    }
    const double em = exp(m);
    out[0] = em * (ch + sh * h);
    out[1] = em * (sh * b);
    out[2] = em * (sh * c);
    out[3] = em * (ch - sh * h);
}

/* Matrix exponential of a 3x3 matrix: scaling by 2^-s until the norm is below 1/2, Taylor series
 * to machine precision, then s squarings. */
static void expm3(const double* K, double* out) {
    double nrm = 0.0;
    for (int i = 0; i < 9; ++i) nrm += fabs(K[i]);
    int s = 0;
    while (nrm > 0.5) { nrm *= 0.5; ++s; }
    const double scale = ldexp(1.0, -s);
    double A[9], term[9], tmp[9];
    for (int i = 0; i < 9; ++i) A[i] = K[i] * scale;
    mat_identity(3, out);
    mat_identity(3, term);
    for (int n = 1; n < 40; ++n) {
        mat_mul(3, term, A, tmp);
        double tn = 0.0;
        for (int i = 0; i < 9; ++i) { term[i] = tmp[i] / n; out[i] += term[i]; tn += fabs(term[i]); }
        if (tn < 1e-20) break;   /* |out| is about 1: below 1e-4 of an ulp */
    }
    for (int k = 0; k < s; ++k) {
        mat_mul(3, out, out, tmp);
        memcpy(out, tmp, sizeof tmp);
    }
}

static void expm_d(int d, const double* K, double* out) {
    if (d == 2) expm2(K, out); else expm3(K, out);
}

/* ------------------------------------------------------------------------------------------ */
/* History of one node: B blocks of at most C points, newest first (Sec. III).                   */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int64_t tp;     /* t': start of the span this point stands for */
    double kap[9];  /* kappa stored with the point (averaged on merge) */
    double F[9];    /* factor over the span: exp(kappa dt) or product of merged factors */
    double gs;      /* strain over the span: gammadot(kappa(t')) dt or sum of merged strains (WM) */
} orc_pt;

typedef struct {
    int d, C, B;
    orc_pt* pts;    /* [B][C]; block index bi = b-1, b = 1 (coarsest) .. B (finest) */
    int* count;     /* [B] */
} orc_hist;

static void hist_init(orc_hist* h, int d, int C, int B) {
    h->d = d; h->C = C; h->B = B;
    h->pts = (orc_pt*)calloc((size_t)B * C, sizeof(orc_pt));
    h->count = (int*)calloc((size_t)B, sizeof(int));
    /* Prefill: every block full of rest points (kappa = 0, factor = 1).  Block B holds t' = -1 ... -C
     * (spacing 1); each coarser block continues backwards with its own spacing 2^(B-b). */
    int64_t tp = 0;
    for (int b = B; b >= 1; --b) {
        const int64_t spacing = (int64_t)1 << (B - b);
        orc_pt* blk = h->pts + (size_t)(b - 1) * C;
        for (int k = 0; k < C; ++k) {
            tp -= spacing;
            blk[k].tp = tp;
            memset(blk[k].kap, 0, sizeof blk[k].kap);
            mat_identity(d, blk[k].F);
            blk[k].gs = 0.0;
        }
        h->count[b - 1] = C;
    }
}

static void hist_free(orc_hist* h) {
    free(h->pts); free(h->count);
    h->pts = NULL; h->count = NULL;
}

/* Insert point p as the newest point of block b (1-based), following the block-merge rule. */
static void hist_insert(orc_hist* h, int b, const orc_pt* p) {
    const int C = h->C, d = h->d;
    orc_pt* blk = h->pts + (size_t)(b - 1) * C;
    if (h->count[b - 1] == C) {
        if (b == 1) {
            h->count[b - 1] -= 1;                 /* coarsest block: the oldest point is dropped */
        } else {
            const orc_pt* o1 = &blk[C - 1];       /* oldest */
            const orc_pt* o2 = &blk[C - 2];       /* second oldest (newer than o1) */
            orc_pt merged;
            memset(&merged, 0, sizeof merged);
            merged.tp = o1->tp;                   /* the merged point keeps the older time */
            for (int i = 0; i < d * d; ++i) merged.kap[i] = 0.5 * (o1->kap[i] + o2->kap[i]);
            mat_mul(d, o2->F, o1->F, merged.F);   /* later factor on the left */
            merged.gs = o1->gs + o2->gs;          /* strain of the joined span */
            h->count[b - 1] -= 2;
            hist_insert(h, b - 1, &merged);
        }
    }
    const int n = h->count[b - 1];
    for (int k = n; k > 0; --k) blk[k] = blk[k - 1];
    blk[0] = *p;
    h->count[b - 1] = n + 1;
}

/* Collect the live points newest-first into out[]; returns their number. */
static int hist_list(const orc_hist* h, orc_pt* out) {
    int n = 0;
    for (int b = h->B; b >= 1; --b) {
        const orc_pt* blk = h->pts + (size_t)(b - 1) * h->C;
        for (int k = 0; k < h->count[b - 1]; ++k) out[n++] = blk[k];
    }
    return n;
}

/* Trapezoidal weights on a sorted (ascending) age grid. */
static void trapezoid_weights(int n, const double* s, double* w) {
    if (n == 1) { w[0] = 0.0; return; }
    for (int k = 0; k < n; ++k) {
        const double lo = (k > 0) ? s[k - 1] : s[k];
        const double hi = (k < n - 1) ? s[k + 1] : s[k];
        w[k] = 0.5 * (hi - lo);
    }
}

enum { ORC_NLM = 0, ORC_INLM = 1, ORC_WM = 2 };
typedef struct { double G_inf, tau, gamma_c; int kind; } orc_model;

/* local shear rate of Sec. II: gammadot^2 = (1/2) tr D^2, D = kappa + kappa^T */
static double shear_rate(int d, const double* K) {
    double trD2 = 0.0;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            const double Dab = K[a * d + b] + K[b * d + a];
            trD2 += Dab * Dab;
        }
    return sqrt(0.5 * trD2);
}

static void pack_sym(int d, const double* S, double* sig) {
    if (d == 2) {
        sig[0] = S[0]; sig[1] = S[3]; sig[2] = S[1];
    } else {
        sig[0] = S[0]; sig[1] = S[4]; sig[2] = S[8];
        sig[3] = S[1]; sig[4] = S[2]; sig[5] = S[5];
    }
}

/*
 * Instantaneous nlM, Eq. (inlM): sigma_struc = G_inf sum_{n>=1} tau_M^n d^(n) with
 * d^(n) = sum_{m=0}^{n} binom(n,m) kappa^m (kappa^T)^(n-m), summed as printed, term by term.  The factor
 * tau_M^n is carried inside the powers, tau_M^n kappa^m (kappa^T)^(n-m) = A^m (A^T)^(n-m) with
 * A = tau_M kappa, so that neither tau_M^n nor kappa^n leaves the double range before the series has
 * converged.  The sum stops once two consecutive terms are below 1e-18 of the partial sum (or vanish:
 * a nilpotent kappa, e.g. simple shear, ends the series at n = 2); after ORC_INLM_NMAX orders without
 * convergence the result is NaN.
 */
#define ORC_INLM_NMAX 1000
static void inlm_stress(int d, const double* K, const orc_model* m, double* sig) {
    const int dd = d * d;
    const double gd = shear_rate(d, K);
    const double rate = 1.0 / m->tau + (isinf(m->gamma_c) ? 0.0 : gd / m->gamma_c);
    const double tM = 1.0 / rate;
    double A[9], AT[9];
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            A[a * d + b] = tM * K[a * d + b];
            AT[a * d + b] = tM * K[b * d + a];
        }
    /* powers A^m and (A^T)^m, m = 0 .. n */
    double* pa = (double*)malloc(sizeof(double) * 9 * (ORC_INLM_NMAX + 1));
    double* pat = (double*)malloc(sizeof(double) * 9 * (ORC_INLM_NMAX + 1));
    mat_identity(d, pa);
    mat_identity(d, pat);
    double S[9] = {0}, term[9], prod[9];
    int quiet = 0, converged = 0;
    for (int n = 1; n <= ORC_INLM_NMAX && !converged; ++n) {
        mat_mul(d, pa + 9 * (n - 1), A, pa + 9 * n);
        mat_mul(d, pat + 9 * (n - 1), AT, pat + 9 * n);
        for (int i = 0; i < dd; ++i) term[i] = 0.0;
        double binom = 1.0;   /* binom(n, mm) */
        for (int mm = 0; mm <= n; ++mm) {
            mat_mul(d, pa + 9 * mm, pat + 9 * (n - mm), prod);
            for (int i = 0; i < dd; ++i) term[i] += binom * prod[i];
            binom = binom * (double)(n - mm) / (double)(mm + 1);
        }
        double tn = 0.0, sn = 0.0;
        for (int i = 0; i < dd; ++i) {
            S[i] += term[i];
            tn = fmax(tn, fabs(term[i]));
            sn = fmax(sn, fabs(S[i]));
        }
        if (!isfinite(tn)) break;
        quiet = (tn <= 1e-18 * sn) ? quiet + 1 : 0;
        if (quiet >= 2) converged = 1;
    }
    free(pa);
    free(pat);
    double out[9];
    for (int i = 0; i < dd; ++i) out[i] = converged ? m->G_inf * S[i] : NAN;
    pack_sym(d, out, sig);
}

/*
 * One history step of one node at time t with the node's velocity gradient kappa_t:
 * insert the new point (Sec. III), re-form E for every retained point from the stored factors
 * (Eq. (eeval)), form -d_{t'}B and the nlM modulus (Eq. (nlmax)) and sum them with the trapezoidal
 * rule into sigma_struc (Eq. (gitt)).  sig receives 3 (2D) or 6 (3D) components.
 */
static void hist_step(orc_hist* h, int64_t t, const double* kappa_t, const orc_model* m,
                      orc_pt* list, double* ages, double* wts, double* sig) {
    const int d = h->d;
    orc_pt p;
    memset(&p, 0, sizeof p);
    p.tp = t;
    memcpy(p.kap, kappa_t, sizeof(double) * d * d);
    expm_d(d, kappa_t, p.F);
    p.gs = shear_rate(d, kappa_t);   /* strain of the step [t, t+1] at the rate of kappa(t) */
    hist_insert(h, h->B, &p);

    const int n = hist_list(h, list);
    for (int k = 0; k < n; ++k) ages[k] = (double)(t - list[k].tp);
    trapezoid_weights(n, ages, wts);

    double S_acc[9] = {0};
    double P[9], Pn[9], M[9], T1[9];
    double strain = 0.0;     /* WM: strain accumulated from t'_k to t, the sum of the spans' strains */
    mat_identity(d, P);
    const double inv_gc = isinf(m->gamma_c) ? 0.0 : 1.0 / m->gamma_c;
    for (int k = 0; k < n; ++k) {
        if (k >= 1) {            /* E_k = F_1 F_2 ... F_k  (E_0 = 1 for the point created now) */
            mat_mul(d, P, list[k].F, Pn);
            memcpy(P, Pn, sizeof(double) * d * d);
            strain += list[k].gs;
        }
        const double* K = list[k].kap;
        mat_mul(d, P, K, T1);        /* E kappa */
        mat_mul_bt(d, T1, P, M);     /* E kappa E^T */
        const double s = ages[k];
        /* Eq. (nlmax): (t - t') gammadot(t') with gammadot from the stored kappa; WM: the strain */
        const double x2 = (m->kind == ORC_WM) ? strain : s * shear_rate(d, K);
        const double G = m->G_inf * exp(-s / m->tau - x2 * inv_gc);
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) S_acc[a * d + b] += wts[k] * G * (M[a * d + b] + M[b * d + a]);
    }
    pack_sym(d, S_acc, sig);
}

/* ------------------------------------------------------------------------------------------ */
/* History-only driver: prescribed kappa sequence, many nodes (test hook for the history sweep).  */
/* ------------------------------------------------------------------------------------------ */

/*
 * kappa_seq: [T][nnodes][d*d], the gradient of step t (t = 0 .. T-1) at every node.
 * sigma_out: [T][nnodes][nsig] (nsig = 3 or 6), sigma_struc after each step; may be NULL except for
 *            the last step when last_only != 0, then it is [nnodes][nsig].
 * model: ORC_NLM, ORC_INLM (no history: sigma from kappa(t) alone) or ORC_WM.
 */
int orc_history_run(int d, int nnodes, int C, int B, double G_inf, double tau, double gamma_c,
                    int T, const double* kappa_seq, double* sigma_out, int last_only, int model) {
    if ((d != 2 && d != 3) || nnodes < 0 || C < 2 || B < 1 || T < 0) return -1;
    if (model != ORC_NLM && model != ORC_INLM && model != ORC_WM) return -1;
    const int nsig = (d == 2) ? 3 : 6;
    const int dd = d * d;
    orc_model m = {G_inf, tau, gamma_c, model};
#pragma omp parallel num_threads(orc_nthreads)
    {
        /* scratch of the node being stepped, one set per thread */
        orc_pt* list = (orc_pt*)malloc(sizeof(orc_pt) * (size_t)B * C);
        double* ages = (double*)malloc(sizeof(double) * (size_t)B * C);
        double* wts = (double*)malloc(sizeof(double) * (size_t)B * C);
#pragma omp for schedule(dynamic, 1)
        for (int node = 0; node < nnodes; ++node) {
            orc_hist h;
            hist_init(&h, d, C, B);
            for (int t = 0; t < T; ++t) {
                double sig[6];
                const double* kt = kappa_seq + ((size_t)t * nnodes + node) * dd;
                if (model == ORC_INLM) inlm_stress(d, kt, &m, sig);
                else hist_step(&h, t, kt, &m, list, ages, wts, sig);
                double* dst = NULL;
                if (!last_only) dst = sigma_out + ((size_t)t * nnodes + node) * nsig;
                else if (t == T - 1) dst = sigma_out + (size_t)node * nsig;
                if (dst) memcpy(dst, sig, sizeof(double) * nsig);
            }
            hist_free(&h);
        }
        free(list); free(ages); free(wts);
    }
    return 0;
}

/* Eq. (inlM) for one gradient (test access): sig receives 3 (2D) or 6 (3D) components. */
int orc_inlm(int d, const double* K, double G_inf, double tau, double gamma_c, double* sig) {
    if (d != 2 && d != 3) return -1;
    orc_model m = {G_inf, tau, gamma_c, ORC_INLM};
    inlm_stress(d, K, &m, sig);
    return 0;
}

/*
 * The retained points of the history grid after step t (all nodes share them): their t' newest
 * first and their trapezoidal weights.  Returns the number of points (<= B*C).
 */
int orc_schedule(int C, int B, int64_t t, int64_t* tp_out, double* w_out) {
    if (C < 2 || B < 1 || t < 0) return -1;
    orc_hist h;
    hist_init(&h, 2, C, B);
    orc_pt* list = (orc_pt*)malloc(sizeof(orc_pt) * (size_t)B * C);
    double* ages = (double*)malloc(sizeof(double) * (size_t)B * C);
    double kz[4] = {0, 0, 0, 0};
    orc_pt p;
    for (int64_t s = 0; s <= t; ++s) {
        memset(&p, 0, sizeof p);
        p.tp = s;
        memcpy(p.kap, kz, sizeof kz);
        mat_identity(2, p.F);
        hist_insert(&h, B, &p);
    }
    const int n = hist_list(&h, list);
    for (int k = 0; k < n; ++k) { tp_out[k] = list[k].tp; ages[k] = (double)(t - list[k].tp); }
    trapezoid_weights(n, ages, w_out);
    free(list); free(ages);
    hist_free(&h);
    return n;
}

/* ------------------------------------------------------------------------------------------ */
/* Lattice-Boltzmann channel (Sec. III): D2Q9 or D3Q19, BGK, forcing Eq. (bodyforce).           */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int d, Q;
    int nx, ny, nz;
    int wall_z;              /* 3D: walls also at z = -1/2 and nz - 1/2 (square duct) */
    double tau_lb, rho0, g[3];
    orc_model m;
    int C, B, trace_full;
    int xbc_pressure;        /* 1: pressure-step boundary along x (ghosts on the linear pressure profile) */
    double dp;               /* pressure drop over one period along x */
    int64_t t;               /* index of the next step */
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    int opp[ORC_MAXQ];
    double* n;               /* [N][Q] population deviations n - w rho0 after streaming, time t */
    double* n_next;
    double* rho_raw;         /* [N] */
    double* j;               /* [N][3] sum c n + f/2 */
    double* u_raw;           /* [N][3] */
    double* rho;             /* [N] fields of the last completed step */
    double* u;               /* [N][3] */
    double* sigma;           /* [N][6] */
    double* kappa;           /* [N][9] */
    double* tr_prev;         /* [N] tr sigma of the previous step */
    orc_hist* hist;          /* [N] */
} orc_channel;

static void set_lattice(orc_channel* ch) {
    if (ch->d == 2) {
        /* D2Q9: rest, four axis links (weight 1/9), four diagonals (1/36), rest weight 4/9 */
        static const int c2[9][2] = {{0,0},{1,0},{0,1},{-1,0},{0,-1},{1,1},{-1,1},{-1,-1},{1,-1}};
        ch->Q = 9;
        for (int i = 0; i < 9; ++i) {
            ch->c[i][0] = c2[i][0]; ch->c[i][1] = c2[i][1]; ch->c[i][2] = 0;
            ch->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else {
        /* D3Q19: rest (1/3), six faces (1/18), twelve edges (1/36) */
        int i = 0;
        ch->c[i][0] = ch->c[i][1] = ch->c[i][2] = 0; ch->w[i++] = 1.0 / 3.0;
        for (int a = 0; a < 3; ++a)
            for (int sgn = 1; sgn >= -1; sgn -= 2) {
                ch->c[i][0] = ch->c[i][1] = ch->c[i][2] = 0;
                ch->c[i][a] = sgn; ch->w[i++] = 1.0 / 18.0;
            }
        for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b)
                for (int sa = 1; sa >= -1; sa -= 2)
                    for (int sb = 1; sb >= -1; sb -= 2) {
                        ch->c[i][0] = ch->c[i][1] = ch->c[i][2] = 0;
                        ch->c[i][a] = sa; ch->c[i][b] = sb; ch->w[i++] = 1.0 / 36.0;
                    }
        ch->Q = 19;
    }
    for (int i = 0; i < ch->Q; ++i)
        for (int k = 0; k < ch->Q; ++k)
            if (ch->c[k][0] == -ch->c[i][0] && ch->c[k][1] == -ch->c[i][1] && ch->c[k][2] == -ch->c[i][2])
                ch->opp[i] = k;
}

static int64_t nodes_of(const orc_channel* ch) { return (int64_t)ch->nx * ch->ny * ch->nz; }

void orc_destroy(orc_channel* ch);

/*
 * Create a channel.  lattice = 9 (D2Q9, nz must be 1, walls in y) or 19 (D3Q19, walls in y, and in z
 * when wall_z).  rho_init: optional [N] initial densities (fluid at rest, n_i = w_i rho).
 */
orc_channel* orc_create(int lattice, int nx, int ny, int nz, int wall_z, double tau_lb, double rho0,
                        double G_inf, double tau, double gamma_c, const double* g, int C, int B,
                        int trace_full, const double* rho_init) {
    if (lattice != 9 && lattice != 19) return NULL;
    if (nx < 1 || ny < 2 || nz < 1 || C < 2 || B < 1 || tau_lb <= 0.5) return NULL;
    if (lattice == 9 && nz != 1) return NULL;
    if (lattice == 19 && wall_z && nz < 2) return NULL;
    orc_channel* ch = (orc_channel*)calloc(1, sizeof(orc_channel));
    ch->d = (lattice == 9) ? 2 : 3;
    ch->nx = nx; ch->ny = ny; ch->nz = nz; ch->wall_z = (lattice == 19) ? wall_z : 0;
    ch->tau_lb = tau_lb; ch->rho0 = rho0;
    ch->g[0] = g ? g[0] : 0.0; ch->g[1] = g ? g[1] : 0.0; ch->g[2] = g ? g[2] : 0.0;
    ch->m.G_inf = G_inf; ch->m.tau = tau; ch->m.gamma_c = gamma_c; ch->m.kind = ORC_NLM;
    ch->C = C; ch->B = B; ch->trace_full = trace_full;
    ch->t = 0;
    set_lattice(ch);
    const int64_t N = nodes_of(ch);
    const int Q = ch->Q;
    ch->n = (double*)calloc((size_t)N * Q, sizeof(double));
    ch->n_next = (double*)calloc((size_t)N * Q, sizeof(double));
    ch->rho_raw = (double*)calloc((size_t)N, sizeof(double));
    ch->j = (double*)calloc((size_t)N * 3, sizeof(double));
    ch->u_raw = (double*)calloc((size_t)N * 3, sizeof(double));
    ch->rho = (double*)calloc((size_t)N, sizeof(double));
    ch->u = (double*)calloc((size_t)N * 3, sizeof(double));
    ch->sigma = (double*)calloc((size_t)N * 6, sizeof(double));
    ch->kappa = (double*)calloc((size_t)N * 9, sizeof(double));
    ch->tr_prev = (double*)calloc((size_t)N, sizeof(double));
    ch->hist = (orc_hist*)calloc((size_t)N, sizeof(orc_hist));
    for (int64_t k = 0; k < N; ++k) hist_init(&ch->hist[k], ch->d, C, B);
    for (int64_t k = 0; k < N; ++k) {
        const double r = rho_init ? rho_init[k] : rho0;
        for (int i = 0; i < Q; ++i) ch->n[k * Q + i] = ch->w[i] * (r - rho0);
        ch->rho[k] = r;
    }
    return ch;
}

void orc_destroy(orc_channel* ch) {
    if (!ch) return;
    const int64_t N = nodes_of(ch);
    for (int64_t k = 0; k < N; ++k) hist_free(&ch->hist[k]);
    free(ch->hist); free(ch->n); free(ch->n_next); free(ch->rho_raw); free(ch->j); free(ch->u_raw);
    free(ch->rho); free(ch->u); free(ch->sigma); free(ch->kappa); free(ch->tr_prev);
    free(ch);
}

/* Pressure-step boundary along x: enabled = 0 restores the plain periodic boundary. */
void orc_set_pressure(orc_channel* ch, int enabled, double dp) {
    ch->xbc_pressure = enabled;
    ch->dp = dp;
}

void orc_set_force(orc_channel* ch, const double* g) {
    ch->g[0] = g[0]; ch->g[1] = g[1]; ch->g[2] = g[2];
}

void orc_set_params(orc_channel* ch, double G_inf, double tau, double gamma_c) {
    ch->m.G_inf = G_inf; ch->m.tau = tau; ch->m.gamma_c = gamma_c;
}

/* Constitutive model of sigma_struc (ORC_NLM, ORC_INLM, ORC_WM); set before the first step. */
int orc_set_model(orc_channel* ch, int kind) {
    if (kind != ORC_NLM && kind != ORC_INLM && kind != ORC_WM) return -1;
    if (ch->t != 0) return -1;
    ch->m.kind = kind;
    return 0;
}

int64_t orc_time(const orc_channel* ch) { return ch->t; }

static int64_t node_id(const orc_channel* ch, int x, int y, int z) {
    return (int64_t)x + (int64_t)ch->nx * ((int64_t)y + (int64_t)ch->ny * z);
}

/*
 * Second-order derivative along one axis of the field f (stride 3 per node, component comp), at
 * coordinate i on an axis of n nodes: central difference if periodic; at a wall-adjacent node the
 * derivative of the parabola through the wall (value 0, half a node away), the node and its inner
 * neighbour: at the low wall (-1/2, 0, 1): f0 + f1/3; at the high wall mirrored.
 */
static double axis_derivative(const double* f_m1, const double* f_0, const double* f_p1, int i, int n,
                              int periodic) {
    if (periodic) return 0.5 * (*f_p1 - *f_m1);
    if (i == 0) return *f_0 + *f_p1 / 3.0;
    if (i == n - 1) return -(*f_0 + *f_m1 / 3.0);
    return 0.5 * (*f_p1 - *f_m1);
}

/* kappa[a][b] = d u_a / d x_b at every node from u (N x 3), Sec. III ("second-order finite
 * difference scheme") with the wall stencil above. */
static void compute_kappa(const orc_channel* ch, const double* u, double* kappa) {
    const int d = ch->d;
#pragma omp parallel for collapse(2) num_threads(orc_nthreads) schedule(static)
    for (int z = 0; z < ch->nz; ++z)
        for (int y = 0; y < ch->ny; ++y)
            for (int x = 0; x < ch->nx; ++x) {
                const int64_t id = node_id(ch, x, y, z);
                for (int b = 0; b < d; ++b) {
                    int64_t im, ip;
                    int i, n, periodic;
                    if (b == 0) {
                        i = x; n = ch->nx; periodic = 1;
                        im = node_id(ch, (x - 1 + n) % n, y, z); ip = node_id(ch, (x + 1) % n, y, z);
                    } else if (b == 1) {
                        i = y; n = ch->ny; periodic = 0;
                        im = node_id(ch, x, y > 0 ? y - 1 : y, z);
                        ip = node_id(ch, x, y < n - 1 ? y + 1 : y, z);
                    } else {
                        i = z; n = ch->nz; periodic = !ch->wall_z;
                        if (periodic) {
                            im = node_id(ch, x, y, (z - 1 + n) % n); ip = node_id(ch, x, y, (z + 1) % n);
                        } else {
                            im = node_id(ch, x, y, z > 0 ? z - 1 : z);
                            ip = node_id(ch, x, y, z < n - 1 ? z + 1 : z);
                        }
                    }
                    for (int a = 0; a < d; ++a)
                        kappa[id * 9 + a * d + b] =
                            axis_derivative(&u[im * 3 + a], &u[id * 3 + a], &u[ip * 3 + a], i, n, periodic);
                }
            }
}

/* Equilibrium (second order in u), Sec. III: w_i rho (1 + c.u/cs2 + (c_a c_b - cs2 delta_ab) u_a u_b/(2 cs2^2)),
 * returned as the deviation from w_i rho0 (drho = rho - rho0), written so that no O(1) terms cancel. */
static double n_eq_dev(const orc_channel* ch, int i, double drho, double rho, const double* u) {
    const double cs2 = 1.0 / 3.0;
    double cu = 0.0, uu = 0.0;
    for (int a = 0; a < ch->d; ++a) { cu += ch->c[i][a] * u[a]; uu += u[a] * u[a]; }
    return ch->w[i] * (drho + rho * (cu / cs2 + (cu * cu - cs2 * uu) / (2.0 * cs2 * cs2)));
}

/*
 * Collision of one node (Sec. III): population deviations n - w rho0 (time t, after streaming),
 * sigma_struc(t) (nsig packed), tr sigma(t-1).  Trace split, density source, fields of Eq. (hydrofields), BGK relaxation to
 * the second-order equilibrium and the forcing term of Eq. (bodyforce).  Writes post[Q], the
 * hydrodynamic rho and u, and tr sigma(t).
 */
static void collide_node(const orc_channel* ch, const double* n, const double* sg, double tr_prev,
                         double* post, double* rho_out, double* u_out, double* tr_out, double* drho_out) {
    const int d = ch->d, Q = ch->Q;
    const double cs2 = 1.0 / 3.0;
    const double f[3] = {ch->rho0 * ch->g[0], ch->rho0 * ch->g[1], ch->rho0 * ch->g[2]};
    double drho_raw = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        drho_raw += n[i];
        for (int a = 0; a < 3; ++a) j[a] += ch->c[i][a] * n[i];
    }
    for (int a = 0; a < 3; ++a) j[a] += 0.5 * f[a];
    double S[3][3] = {{0}};
    if (d == 2) {
        S[0][0] = sg[0]; S[1][1] = sg[1]; S[0][1] = S[1][0] = sg[2];
    } else {
        S[0][0] = sg[0]; S[1][1] = sg[1]; S[2][2] = sg[2];
        S[0][1] = S[1][0] = sg[3]; S[0][2] = S[2][0] = sg[4]; S[1][2] = S[2][1] = sg[5];
    }
    double tr = 0.0;
    for (int a = 0; a < d; ++a) tr += S[a][a];
    double dt_drho = 0.0;
    if (ch->trace_full) dt_drho = -(tr - tr_prev) / ((double)d * cs2);
    const double drho = drho_raw + 0.5 * dt_drho;     /* rho - rho0 */
    const double rho = ch->rho0 + drho;
    double u[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) u[a] = j[a] / rho;
    double Sb[3][3];   /* traceless part */
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Sb[a][b] = S[a][b] - ((a == b) ? tr / d : 0.0);
    for (int i = 0; i < Q; ++i) {
        const double neq = n_eq_dev(ch, i, drho, rho, u);
        /* Eq. (bodyforce) */
        double stress = 0.0, guo2 = 0.0, cf = 0.0;
        for (int a = 0; a < d; ++a) {
            cf += ch->c[i][a] * f[a];
            for (int b = 0; b < d; ++b) {
                const double Lab = ch->c[i][a] * ch->c[i][b] - ((a == b) ? cs2 : 0.0);
                stress += Sb[a][b] * Lab;
                guo2 += Lab * (-dt_drho * u[a] * u[b] + u[b] * f[a] + u[a] * f[b]);
            }
        }
        const double Fi = ch->w[i] * (-stress / (2.0 * cs2 * cs2 * ch->tau_lb) +
                                      (1.0 - 0.5 / ch->tau_lb) *
                                          (dt_drho + cf / cs2 + guo2 / (2.0 * cs2 * cs2)));
        post[i] = n[i] - (n[i] - neq) / ch->tau_lb + Fi;
    }
    *rho_out = rho;
    *drho_out = drho;
    for (int a = 0; a < 3; ++a) u_out[a] = u[a];
    *tr_out = tr;
}

/* One full hybrid step t -> t+1. */
static void channel_step(orc_channel* ch) {
    const int d = ch->d, Q = ch->Q;
    const int64_t N = nodes_of(ch);
    const double f[3] = {ch->rho0 * ch->g[0], ch->rho0 * ch->g[1], ch->rho0 * ch->g[2]};

    /* 1. raw moments: rho_raw = sum n, j = sum c n + f/2, u_raw = j / rho_raw
     *    (sum w rho0 = rho0 and sum c w rho0 = 0 for the stored deviations) */
#pragma omp parallel for num_threads(orc_nthreads) schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        double dr = 0.0, jj[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            const double ni = ch->n[k * Q + i];
            dr += ni;
            for (int a = 0; a < 3; ++a) jj[a] += ch->c[i][a] * ni;
        }
        const double r = ch->rho0 + dr;
        ch->rho_raw[k] = r;
        for (int a = 0; a < 3; ++a) {
            ch->j[k * 3 + a] = jj[a] + 0.5 * f[a];
            ch->u_raw[k * 3 + a] = (a < d) ? ch->j[k * 3 + a] / r : 0.0;
        }
    }
    /* 2. kappa(t) by finite differences of u_raw */
    compute_kappa(ch, ch->u_raw, ch->kappa);
    /* 3-4. history: sigma_struc(t) */
#pragma omp parallel num_threads(orc_nthreads)
    {
        /* scratch of the node being stepped, one set per thread */
        const size_t L = (size_t)ch->B * ch->C;
        orc_pt* list = (orc_pt*)malloc(sizeof(orc_pt) * L);
        double* ages = (double*)malloc(sizeof(double) * L);
        double* wts = (double*)malloc(sizeof(double) * L);
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < N; ++k) {
            double kap[9];
            for (int i = 0; i < d * d; ++i) kap[i] = ch->kappa[k * 9 + i];
            if (ch->m.kind == ORC_INLM) inlm_stress(d, kap, &ch->m, &ch->sigma[k * 6]);
            else hist_step(&ch->hist[k], ch->t, kap, &ch->m, list, ages, wts, &ch->sigma[k * 6]);
        }
        free(list); free(ages); free(wts);
    }
    /* 5-7. trace split, density source, collision with forcing, streaming (every destination population
     * is written by exactly one source node, so rows may run on different threads) */
    memset(ch->n_next, 0, sizeof(double) * (size_t)N * Q);
#pragma omp parallel for collapse(2) num_threads(orc_nthreads) schedule(static)
    for (int z = 0; z < ch->nz; ++z)
        for (int y = 0; y < ch->ny; ++y)
            for (int x = 0; x < ch->nx; ++x) {
                const int64_t k = node_id(ch, x, y, z);
                double post[ORC_MAXQ], rho, u[3], tr, drho;
                collide_node(ch, &ch->n[k * Q], &ch->sigma[k * 6], ch->tr_prev[k], post, &rho, u, &tr, &drho);
                for (int i = 0; i < Q; ++i) {
                    /* stream with half-way bounce-back */
                    int xd = x + ch->c[i][0], yd = y + ch->c[i][1], zd = z + ch->c[i][2];
                    xd = (xd + ch->nx) % ch->nx;
                    int wall = (yd < 0 || yd >= ch->ny);
                    if (d == 3) {
                        if (ch->wall_z) wall = wall || (zd < 0 || zd >= ch->nz);
                        else zd = (zd + ch->nz) % ch->nz;
                    }
                    double val = post[i];
                    const int xs = x + ch->c[i][0];
                    if (!wall && ch->xbc_pressure && (xs < 0 || xs >= ch->nx)) {
                        /* crossing the seam: the population of the ghost image (inlet ghost for +x,
                         * outlet ghost for -x) -- equilibrium at the ghost density, this node's
                         * non-equilibrium part, both as deviations from w rho0 (the deviations of the
                         * ghost and node densities from rho0 taken as such, not as rho - rho0) */
                        const double half = 0.5 * 3.0 * ch->dp * (ch->nx + 1.0) / ch->nx;
                        const double drho_gh = (xs >= ch->nx) ? half : -half;
                        val = n_eq_dev(ch, i, drho_gh, ch->rho0 + drho_gh, u) +
                              (post[i] - n_eq_dev(ch, i, drho, rho, u));
                    }
                    if (wall) ch->n_next[k * Q + ch->opp[i]] = val;
                    else ch->n_next[node_id(ch, xd, yd, zd) * Q + i] = val;
                }
                ch->rho[k] = rho;
                for (int a = 0; a < 3; ++a) ch->u[k * 3 + a] = u[a];
                ch->tr_prev[k] = ch->trace_full ? tr : 0.0;
            }
    double* tmp = ch->n; ch->n = ch->n_next; ch->n_next = tmp;
    ch->t += 1;
}

int orc_step(orc_channel* ch, int64_t nsteps) {
    for (int64_t s = 0; s < nsteps; ++s) channel_step(ch);
    return 0;
}

/*
 * Fields of the last completed step, each [N][...] in node order (any pointer may be NULL):
 * rho [N]; u [N][d]; sigma_struc [N][nsig]; kappa [N][d*d]; n1 = sigma_xx - sigma_yy [N].
 */
void orc_fields(const orc_channel* ch, double* rho, double* u, double* sigma, double* kappa, double* n1) {
    const int d = ch->d, nsig = (d == 2) ? 3 : 6;
    const int64_t N = nodes_of(ch);
    for (int64_t k = 0; k < N; ++k) {
        if (rho) rho[k] = ch->rho[k];
        if (u) for (int a = 0; a < d; ++a) u[k * d + a] = ch->u[k * 3 + a];
        if (sigma) for (int c = 0; c < nsig; ++c) sigma[k * nsig + c] = ch->sigma[k * 6 + c];
        if (kappa) for (int c = 0; c < d * d; ++c) kappa[k * d * d + c] = ch->kappa[k * 9 + c];
        if (n1) n1[k] = ch->sigma[k * 6 + 0] - ch->sigma[k * 6 + 1];
    }
}

/* Populations [N][Q] after the last streaming (time t). */
void orc_populations(const orc_channel* ch, double* out) {
    const int64_t N = nodes_of(ch);
    for (int64_t k = 0; k < N; ++k)
        for (int i = 0; i < ch->Q; ++i) out[k * ch->Q + i] = ch->w[i] * ch->rho0 + ch->n[k * ch->Q + i];
}

/*
 * Mass bookkeeping: total sum of populations, and the sum of the pressure-equivalent density
 * delta rho(t-1) = -tr sigma(t-1)/(d c_s^2) held back by the density source.
 */
void orc_mass(const orc_channel* ch, double* sum_n, double* sum_drho_prev) {
    const int64_t N = nodes_of(ch);
    double s = 0.0, r = 0.0;
    for (int64_t k = 0; k < N * ch->Q; ++k) s += ch->n[k];
    for (int64_t k = 0; k < N; ++k) r += -ch->tr_prev[k] / ((double)ch->d / 3.0);
    *sum_n = s + ch->rho0 * (double)N;   /* sum of w rho0 over the lattice is rho0 per node */
    *sum_drho_prev = r;
}

/* kappa from a prescribed velocity field u [N][3] (test access to the finite-difference stencil). */
void orc_kappa_of(const orc_channel* ch, const double* u, double* kappa_out) {
    const int d = ch->d;
    const int64_t N = nodes_of(ch);
    double* K = (double*)malloc(sizeof(double) * (size_t)N * 9);
    compute_kappa(ch, u, K);
    for (int64_t k = 0; k < N; ++k)
        for (int c = 0; c < d * d; ++c) kappa_out[k * d * d + c] = K[k * 9 + c];
    free(K);
}

/* exp of a d x d matrix (test access). */
void orc_expm(int d, const double* K, double* out) { expm_d(d, K, out); }

/* Collision of one node with the channel's parameters (test access to Eq. (bodyforce)): full
 * populations n in, full post-collision populations out. */
void orc_collide(const orc_channel* ch, const double* n, const double* sigma, double tr_prev, double* post,
                 double* rho, double* u) {
    double tr, drho, dn[ORC_MAXQ];
    for (int i = 0; i < ch->Q; ++i) dn[i] = n[i] - ch->w[i] * ch->rho0;
    collide_node(ch, dn, sigma, tr_prev, post, rho, u, &tr, &drho);
    for (int i = 0; i < ch->Q; ++i) post[i] += ch->w[i] * ch->rho0;
}
