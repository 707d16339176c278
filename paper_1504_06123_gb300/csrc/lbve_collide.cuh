// lbve_collide.cuh -- the per-node collision kernel of the hybrid LB step (Sec. III of arXiv:1504.06123),
// the history-free stress of the instantaneous nlM (Eq. inlM), and the field gather / reduction kernels.
//
//   k_collide_stream : per node: kappa(t) by finite differences, sigma_struc(t) (the history commit of
//                      lbve_kernels.cuh, or Eq. (inlM) on kappa(t)), trace split, density source, BGK
//                      collision with the forcing of Eq. (bodyforce), push streaming with half-way
//                      bounce-back.
#pragma once
#include "lbve_kernels.cuh"

namespace lbk {

// ------------------------------------------------------------------------------------------------
// Instantaneous nlM, Eq. (inlM): no history.  sigma_struc(t) = G_inf sum_{n>=1} tau_M^n d^(n)[kappa(t)],
// tau_M = (1/tau + gammadot(t)/gamma_c)^-1.  The d^(n) are the Taylor coefficients of
// exp(kappa s) exp(kappa^T s), so d^(1) = D and d^(n+1) = kappa d^(n) + d^(n) kappa^T: with A = tau_M kappa
// the terms T_n = tau_M^n d^(n) follow T_1 = tau_M D, T_{n+1} = A T_n + T_n A^T, summed in the arithmetic
// type T until two consecutive terms are below 1e-18 of the partial sum (a nilpotent kappa, simple shear,
// ends the series at n = 2).  NaN when the series has not converged after kInlmTerms terms or overflows:
// Eq. (inlM) then has no sum (no steady state).  The stopping rule is the same in both arithmetic types,
// so FP32 and FP64 agree on where the sum exists.
// ------------------------------------------------------------------------------------------------
template <typename T> struct Instant { int B, C; };   // B = 1, C = 4: the shared schedule code is unused
constexpr int kInlmTerms = 1000;
constexpr double kInlmEps = 1e-18;

// Packed symmetric components: xx, yy, xy (2D); xx, yy, zz, xy, xz, yz (3D).
template <int D> __device__ __forceinline__ constexpr int sym_r(int i) { return D == 2 ? (i == 1 ? 1 : 0) : (i < 3 ? i : (i == 5 ? 1 : 0)); }
template <int D> __device__ __forceinline__ constexpr int sym_c(int i) { return D == 2 ? (i == 0 ? 0 : 1) : (i < 3 ? i : (i == 3 ? 1 : 2)); }

template <int D, typename T, typename N>
__device__ __forceinline__ void inlm_stress(const double* ktd, const Chan& p, N* sig) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    const double tMd = 1.0 / (p.inv_tau + shear_rate_d<D>(ktd) * p.inv_gc);
    T A[DD], Tn[NS], Z[NS];   // Tn and Z symmetric, packed
#pragma unroll
    for (int i = 0; i < DD; ++i) A[i] = (T)(tMd * ktd[i]);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int r = sym_r<D>(i), c = sym_c<D>(i);
        Tn[i] = (T)(tMd * (ktd[r * D + c] + ktd[c * D + r]));
        Z[i] = Tn[i];
    }
    bool ok = false;
    int quiet = 0;
    for (int n = 2; n <= kInlmTerms; ++n) {
        T Tm[DD];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int r = sym_r<D>(i), c = sym_c<D>(i);
            Tm[r * D + c] = Tm[c * D + r] = Tn[i];
        }
        T P[DD];   // A T_n
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                T s = A[r * D] * Tm[c];
#pragma unroll
                for (int k = 1; k < D; ++k) s += A[r * D + k] * Tm[k * D + c];
                P[r * D + c] = s;
            }
        T tn = 0, zn = 0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {   // T_{n+1} = A T_n + (A T_n)^T
            const int r = sym_r<D>(i), c = sym_c<D>(i);
            const T v = P[r * D + c] + P[c * D + r];
            Tn[i] = v;
            Z[i] += v;
            tn = fmax(tn, fabs(v));
            zn = fmax(zn, fabs(Z[i]));
        }
        if (!isfinite(tn) || !isfinite(zn)) break;   // diverged
        quiet = (tn <= T(kInlmEps) * zn) ? quiet + 1 : 0;
        if (quiet >= 2) { ok = true; break; }
    }
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int i = 0; i < NS; ++i) sig[i] = (N)(ok ? p.G_inf * (double)Z[i] : nan);
}

template <int D, typename T, typename N>
__device__ __forceinline__ void hist_commit_any(Arith<N>, const Instant<T>&, const BlockStep*, long long, int,
                                                const double* /*kprev*/, const double* ktd, const Chan& p,
                                                N* sig, long long /*t*/) {
    inlm_stress<D, T, N>(ktd, p, sig);
}

// ------------------------------------------------------------------------------------------------
// K3: collision with the non-Newtonian forcing and push streaming
// ------------------------------------------------------------------------------------------------
template <typename P> struct CollArgs {
    const P* __restrict__ dn_in;        // [Q][Npad]
    P* __restrict__ dn_out;             // [Q][Npad]
    const double* __restrict__ u_raw;   // [D][Npad]  for kappa(t)
    double* __restrict__ sigma;         // [NS][Npad] sigma_struc(t) out
    double* __restrict__ kappa;         // [DD][Npad] kappa(t) out
    double* __restrict__ tr_prev;       // [Npad]
    double* __restrict__ rho;           // [Npad] rho - rho0
    double* __restrict__ u;             // [D][Npad]
    const long long* t_dev;             // step index t
};

// One node per thread: history commit (sigma_struc(t), merges, new point), then the collision with
// that stress and push streaming.  T: arithmetic type of the collision (double for double populations;
// float for float).  The finite-difference gradient and the node scalars run in double, the node fields
// are stored in double.
template <int Q, typename P, typename T, class H>
__global__ void __launch_bounds__(256) k_collide_stream(CollArgs<P> a, H h, Geom g) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    __shared__ BlockStep s_bs[LBVE_MAXB];
    const long long t = *a.t_dev;
    sched_step_cta(h.B, h.C, t, s_bs);
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    const long long Np = g.Npad;
    const Chan& p = g.ch[chan_index(g, n)];
    // N: arithmetic of the gradient, the commit's sums, the moments and the node scalars (trace, density
    // source, rho, u) -- float only with float populations and the 16-bit history, whose storage rounding
    // (2^-15 of a vector's scale) is far coarser, else double.  With float, k_moments stored u_raw in float
    // too.  The node fields are stored in double either way.
    using N = typename std::conditional<sizeof(P) == 4 && Hist16<H>::value, float, double>::type;
    N sg[NS];
    {
        N ktd[DD];
        double kprev[DD];
        kappa_fd<D>(reinterpret_cast<const N*>(a.u_raw), Np, p, n, ktd);
#pragma unroll
        for (int c = 0; c < DD; ++c) kprev[c] = a.kappa[c * Np + n];
        hist_commit_any<D>(Arith<N>(), h, s_bs, Np, n, kprev, ktd, p, sg, t);
#pragma unroll
        for (int i = 0; i < NS; ++i) a.sigma[i * Np + n] = (double)sg[i];
#pragma unroll
        for (int c = 0; c < DD; ++c) a.kappa[c * Np + n] = (double)ktd[c];
    }
    T dn[Q];
    N dm[Q], drho_m, jd_m[3];
#pragma unroll
    for (int q = 0; q < Q; ++q) { dn[q] = (T)a.dn_in[q * Np + n]; dm[q] = (N)a.dn_in[q * Np + n]; }
    node_moments<Q, N>(dm, drho_m, jd_m);
    // stress: traceless part and density source (Sec. III, trace split)
    T S[3][3];
    N trd = 0;
    if (D == 2) {
        S[0][0] = (T)sg[0]; S[1][1] = (T)sg[1];
        S[0][1] = S[1][0] = (T)sg[2];
        trd = sg[0] + sg[1];
    } else {
        S[0][0] = (T)sg[0]; S[1][1] = (T)sg[1]; S[2][2] = (T)sg[2];
        S[0][1] = S[1][0] = (T)sg[3];
        S[0][2] = S[2][0] = (T)sg[4];
        S[1][2] = S[2][1] = (T)sg[5];
        trd = sg[0] + sg[1] + sg[2];
    }
    N ddr_d = 0;   // tr_prev holds the last step's N trace, exactly
    if (p.trace_full) ddr_d = -(trd - (N)a.tr_prev[n]) * N(3.0 / D);   // -(tr - tr_prev)/(d cs^2)
    const N drho_d = drho_m + N(0.5) * ddr_d;                            // rho - rho0
    const N rho_d = chan_val<N>(p.rho0, p.rho0_f) + drho_d;
    const N inv_rho = N(1) / rho_d;
    N ud[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < D; ++c) ud[c] = (jd_m[c] + N(0.5) * chan_val<N>(p.f[c], p.f_f[c])) * inv_rho;
    const T tr = (T)trd, ddr = (T)ddr_d, drho = (T)drho_d, rho = (T)rho_d;
    T u[3], f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) { u[c] = (T)ud[c]; f[c] = chan_val<T>(p.f[c], p.f_f[c]); }
#pragma unroll
    for (int c = 0; c < D; ++c) S[c][c] -= tr * T(1.0 / D);
    T uu = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) uu += u[c] * u[c];
    const T omega = chan_val<T>(p.omega, p.omega_f);
    const T fpre = T(1) - T(0.5) * omega;
    // BGK relaxation to the second-order equilibrium plus the forcing of Eq. (bodyforce), regrouped per
    // node.  With X_ab = -ddr u_a u_b + u_b f_a + u_a f_b (its second-order forcing term), S traceless,
    // 1/cs2 = 3, 1/(2 cs4) = 4.5 and cs2/(2 cs4) = 1.5, every post-collision population is
    //   n*_q = (1 - omega) n_q + w_q (a0 + c_q.v + c_q.M.c_q)
    //   a0 = omega (drho - 1.5 rho u.u) + fpre (ddr - 1.5 tr X)
    //   v  = 3 (omega rho u + fpre f)
    //   M  = 4.5 (omega rho u u^T - omega S + fpre X)
    // i.e. n - omega (n - n_eq) + F with n_eq = w (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)) and
    // F = w (-4.5 omega c.S.c + fpre (ddr + 3 c.f + 4.5 c.X.c - 1.5 tr X)); the node-level terms are
    // formed once instead of once per population.
    const T orho = omega * rho;
    T trX = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) trX += T(2) * u[c] * f[c] - ddr * u[c] * u[c];
    const T a0 = omega * drho - T(1.5) * orho * uu + fpre * (ddr - T(1.5) * trX);
    T v[3], M[3][3];
#pragma unroll
    for (int r = 0; r < D; ++r) {
        v[r] = T(3) * (orho * u[r] + fpre * f[r]);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const T Xrc = -ddr * u[r] * u[c] + u[c] * f[r] + u[r] * f[c];
            M[r][c] = T(4.5) * (orho * u[r] * u[c] - omega * S[r][c] + fpre * Xrc);
        }
    }
    const T keep = T(1) - omega;

    int x, y, z;
    node_xyz(p, n, x, y, z);
    // the channel's geometry in registers: the population stores below may alias the channel table as far
    // as the compiler can tell, which would reload every field after each store
    const int cnx = p.nx, cny = p.ny, cnz = p.nz, coff = p.off;
    const bool cwz = p.wall_z != 0, cxbc = p.xbc != 0;
    const T cdgh = chan_val<T>(p.drho_gh, p.drho_gh_f);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cq[3] = {L::cx(q), L::cy(q), L::cz(q)};
        // c.v and c.M.c with c_q in {-1, 0, 1}: sums and differences only
        T cv = 0, cMc = 0;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            if (cq[r] > 0) cv += v[r];
            if (cq[r] < 0) cv -= v[r];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if (cq[r] && cq[c]) {
                    if (cq[r] * cq[c] > 0) cMc += M[r][c];
                    else cMc -= M[r][c];
                }
            }
        }
        T post_t = keep * dn[q] + (T)L::w(q) * (a0 + cv + cMc);
        // push with half-way bounce-back
        const int xs = x + cq[0];
        const int xd = xs < 0 ? cnx - 1 : (xs >= cnx ? 0 : xs);
        const int yd = y + cq[1];
        bool wall = yd < 0 || yd >= cny;
        int zd = z + cq[2];
        if (D == 3) {
            if (cwz) wall = wall || zd < 0 || zd >= cnz;
            else zd = zd < 0 ? cnz - 1 : (zd >= cnz ? 0 : zd);
        }
        if (cq[0] != 0 && cxbc && !wall && xd != xs) {
            // pressure-step boundary: a population crossing the seam streams from the ghost image
            // n_eq(rho_ghost, u) + (n* - n_eq(rho, u)) = n* + w (rho_ghost - rho)(1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u);
            // the inlet ghost (rho0 + drho_gh) for +x, the outlet ghost (rho0 - drho_gh) for -x
            T cu = 0;
#pragma unroll
            for (int r = 0; r < D; ++r) cu += cq[r] * u[r];
            const T dgh = (cq[0] > 0 ? cdgh : -cdgh) - drho;
            post_t += (T)L::w(q) * dgh * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
        }
        const P post = (P)post_t;
        if (wall) a.dn_out[L::opp(q) * Np + n] = post;
        else a.dn_out[q * Np + (coff + xd + cnx * (yd + cny * zd))] = post;
    }
    a.rho[n] = (double)drho_d;
#pragma unroll
    for (int c = 0; c < D; ++c) a.u[c * Np + n] = (double)ud[c];
    a.tr_prev[n] = p.trace_full ? (double)trd : 0.0;
}

// ------------------------------------------------------------------------------------------------
// Field gather (lbve_fields) and reductions (lbve_mass)
// ------------------------------------------------------------------------------------------------
template <typename real>
__global__ void k_gather(const real* __restrict__ src, long long Npad, int ncomp, int N, double offset,
                         double* __restrict__ dst, int* nonfinite) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)ncomp * N) return;
    const int c = (int)(i / N), n = (int)(i % N);
    const double v = (double)src[c * Npad + n] + offset;
    dst[i] = v;
    if (!isfinite(v)) atomicOr(nonfinite, 1);
}

template <typename real>
__global__ void k_n1(const real* __restrict__ sigma, long long Npad, int N, double* __restrict__ dst,
                     int* nonfinite) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double v = (double)sigma[n] - (double)sigma[Npad + n];
    dst[n] = v;
    if (!isfinite(v)) atomicOr(nonfinite, 1);
}

// Probe recorder (lbve_set_probes): after the step that completes t = t_dev + 1 steps, when t is a
// multiple of `every`, append [t, per probe: rho, u[D], sigma[NS]] as record *cnt (stored while
// *cnt < cap; the count goes on so that the host can see an overflow).  One block; every thread reads
// the count before the barrier, thread 0 advances it after.
__global__ void k_probe(const double* __restrict__ rho, const double* __restrict__ u,
                        const double* __restrict__ sigma, long long Npad, int D, int NS,
                        const long long* __restrict__ nodes, int P, double rho0, const long long* t_dev,
                        int every, long long cap, double* __restrict__ rec, long long* cnt) {
    const long long t = *t_dev + 1;
    if (t % every != 0) return;
    const long long k = *cnt;
    const int PV = 1 + D + NS;
    if (k < cap) {
        double* r = rec + k * (1 + (long long)P * PV);
        for (int i = threadIdx.x; i < P * PV; i += blockDim.x) {
            const int p = i / PV, v = i - p * PV;
            const long long n = nodes[p];
            double x;
            if (v == 0) x = rho[n] + rho0;                       // stored as rho - rho0
            else if (v <= D) x = u[(v - 1) * Npad + n];
            else x = sigma[(v - 1 - D) * Npad + n];
            r[1 + i] = x;
        }
        if (threadIdx.x == 0) r[0] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *cnt = k + 1;
}

template <typename real>
__global__ void k_sum(const real* __restrict__ src, long long Npad, int ncomp, int N, double scale,
                      double* __restrict__ out) {
    double s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)ncomp * N;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / N), n = (int)(i % N);
        s += (double)src[c * Npad + n];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s * scale);
}

}  // namespace lbk
