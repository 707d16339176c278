// lbve_adjoint.cuh -- reverse-mode (adjoint) model of the hybrid step, form "P" history.  The tape (the
// per-step states the forward recorded: populations TP, history TH) is read in its storage precision, FP64
// or FP32; every adjoint quantity and every partial of dL/dtheta is carried in FP64.
//
// For a loss of the fields of the last step, the adjoint runs the steps backwards: lambda of the state
// after step t (populations after streaming, history slots after the commit, tr sigma of step t) gives
// lambda of the state before step t, and every step adds its share of dL/dtheta for
// theta = (G_inf, tau, gamma_c, g_x).  The forward quantities of step t are recomputed per node from the
// state before the step (taped per step inside a checkpoint segment by the runtime).
//
// Five kernels per step (the history parts split over slot chunks like the forward sweep, so that the
// O(nodes x points) work runs on (node, chunk) threads; every chunk's sums are added in chunk order):
//   k_adj_sig    (node, chunk) threads: forward recompute of the history sweep of step t on the taped
//                history -- partial sums of the integrand (the stress before the new point);
//   k_adj_node   one thread per node: forward recompute (moments, kappa(t), sigma from the partial sums,
//                collision), then the adjoint of the collision + streaming (a pull from the neighbours) and
//                of the commit (merges and new point in reverse order); writes the pairing matrix of
//                lambda(sigma_struc) for the sweep's adjoint, lambda of kappa(t) and the node's part of
//                lambda(populations);
//   k_adj_hist   (node, chunk) threads: adjoint of the history sweep (point integrands, in-place advance)
//                with partial sums of lambda(A), lambda(1/tau), lambda(1/gamma_c) per chunk;
//   k_adj_fin    one thread per node: the chunk sums, the adjoint of A = exp(kappa(t-1)) - 1 and the rate
//                parts of dL/dtheta;
//   k_adj_fd     one thread per node: transpose of the finite-difference stencil (gathers lambda kappa(t)
//                from the nodes whose stencil reads this node) and the adjoint of the raw moments.
#pragma once
#include "lbve_kernels.cuh"

namespace lbk {

struct AdjPar {
    double G_inf, tau, gamma_c, inv_tau, inv_gc, rho0, tau_lb, f[3];
    int trace_full;
};

// Adjoint of A = exp(K) - 1 as the forward forms it (expm1_mat: Horner's scheme of the Taylor polynomial of
// order ORDER, 4 for a float history, 8 for double): P_ORDER = K/ORDER, P_m = (K + K P_{m+1})/m for
// m = ORDER-1 .. 1, A = P_1.  Reversed: lambda_K += lambda_{P_m} (1 + P_{m+1})^T / m and
// lambda_{P_{m+1}} = K^T lambda_{P_m} / m, then lambda_K += lambda_{P_ORDER} / ORDER.  In double.
template <int D, int ORDER>
__device__ inline void expm1_adjoint(const double* K, const double* lamA, double* lamK) {
    constexpr int DD = D * D;
    double P[ORDER + 1][DD];   // P[m], m = 1 .. ORDER
#pragma unroll
    for (int i = 0; i < DD; ++i) P[ORDER][i] = K[i] * (1.0 / ORDER);
#pragma unroll
    for (int m = ORDER - 1; m >= 1; --m)
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                double s = K[r * D + c];
#pragma unroll
                for (int k = 0; k < D; ++k) s += K[r * D + k] * P[m + 1][k * D + c];
                P[m][r * D + c] = s * (1.0 / m);
            }
    double lp[DD];
#pragma unroll
    for (int i = 0; i < DD; ++i) lp[i] = lamA[i];
#pragma unroll
    for (int m = 1; m <= ORDER - 1; ++m) {
        double nx[DD];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                double s = lp[r * D + c], t = 0.0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    s += lp[r * D + k] * P[m + 1][c * D + k];   // lambda_{P_m} (1 + P_{m+1})^T
                    t += K[k * D + r] * lp[k * D + c];          // K^T lambda_{P_m}
                }
                lamK[r * D + c] += s * (1.0 / m);
                nx[r * D + c] = t * (1.0 / m);
            }
#pragma unroll
        for (int i = 0; i < DD; ++i) lp[i] = nx[i];
    }
#pragma unroll
    for (int i = 0; i < DD; ++i) lamK[i] += lp[i] * (1.0 / ORDER);
}

// Packed symmetric (NS components) -> full matrix of the adjoint pairing: sum_p lam_p S_p = tr(Lt S)
// with Lt_aa = lam_aa and Lt_ab = lam_ab / 2 off the diagonal.
template <int D>
__device__ inline void packed_to_pairing(const double* lam, double* Lt) {
    if (D == 2) {
        Lt[0] = lam[0]; Lt[3] = lam[1]; Lt[1] = Lt[2] = 0.5 * lam[2];
    } else {
        Lt[0] = lam[0]; Lt[4] = lam[1]; Lt[8] = lam[2];
        Lt[1] = Lt[3] = 0.5 * lam[3]; Lt[2] = Lt[6] = 0.5 * lam[4]; Lt[5] = Lt[7] = 0.5 * lam[5];
    }
}

// Forward integrand (same arithmetic as point_integrand) returning S packed, g and gammadot; and its
// adjoint for a pairing matrix Lt: lamE (dL/dE), lamk (dL/dkappa), and the scalar parts for the rates.
// R: the arithmetic of the history (the forward's exp and sqrt of that type, FastMath); the rate parts are
// accumulated in double.
template <int D, typename R>
__device__ inline void integrand_adjoint(const R* X, const R* kap, R age, R w, R inv_tau, R inv_gc, const R* Lt,
                                         R* lamX, R* lamk, double* lam_inv_tau, double* lam_inv_gc) {
    constexpr int DD = D * D;
    R E[DD];
#pragma unroll
    for (int i = 0; i < DD; ++i) E[i] = X[i] + ((i % (D + 1) == 0) ? R(1) : R(0));
    // M = E kap E^T
    R EK[DD], M[DD];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += E[r * D + k] * kap[k * D + c];
            EK[r * D + c] = s;
        }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += EK[r * D + k] * E[c * D + k];
            M[r * D + c] = s;
        }
    R trD2 = 0, Dm[DD];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            Dm[r * D + c] = kap[r * D + c] + kap[c * D + r];
            trD2 += Dm[r * D + c] * Dm[r * D + c];
        }
    const R gd = FastMath<R>::sqrt_pos(R(0.5) * trD2);
    const R g = FastMath<R>::exp_neg(age * (inv_tau + gd * inv_gc));
    // sS = tr(Lt S), S = M + M^T
    R sS = 0;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) sS += Lt[r * D + c] * (M[c * D + r] + M[r * D + c]);
    // dS: lamE = 2 w g Lt E (kap + kap^T); lamkap = 2 w g E^T Lt E
    R LE[DD];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += Lt[r * D + k] * E[k * D + c];
            LE[r * D + c] = s;
        }
    const R wg2 = R(2) * w * g;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = 0, s2 = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                s += LE[r * D + k] * Dm[k * D + c];          // Lt E (kap + kap^T)
                s2 += E[k * D + r] * LE[k * D + c];          // E^T Lt E
            }
            lamX[r * D + c] += wg2 * s;
            lamk[r * D + c] += wg2 * s2;
        }
    // dg: g = exp(-age (inv_tau + gd inv_gc))
    const R dl_dg = w * sS;
    *lam_inv_tau += (double)(dl_dg * (-age * g));
    *lam_inv_gc += (double)(dl_dg * (-age * gd * g));
    if (gd > R(0)) {
        const R dl_dgd = dl_dg * (-age * inv_gc * g);
#pragma unroll
        for (int i = 0; i < DD; ++i) lamk[i] += dl_dgd * Dm[i] / gd;
    }
}

template <typename TP, typename TH> struct AdjArgs {
    const TP* n;            // [Q][Npad] populations of step t (before collision)
    const TH* X;            // [L][DD][Npad] history before the step
    const TH* K;            // [L][DD][Npad]
    const double* trp;      // [Npad] tr sigma(t-1)
    const double* u_raw;    // [D][Npad] raw velocity of step t (recomputed by k_moments)
    const double* lam_n1;   // [Q][Npad] lambda of the populations after step t
    double* lam_n0;         // [Q][Npad] lambda of the populations before step t (this kernel's part)
    TH* lamX;               // [L][DD][Npad] in: after step t; out: before step t (history type)
    TH* lamK;               // [L][DD][Npad]
    double* lam_trp;        // [Npad] in: lambda of tr sigma(t); out: of tr sigma(t-1)
    double* lam_kt;         // [DD][Npad] out: lambda of kappa(t)
    double* lam_theta;      // [4][Npad] += per-node parts of dL/dtheta
    const double* seed_u;   // [D][Npad] dL/du of this step's velocity (last step), or nullptr
    const double* seed_s;   // [NS][Npad] dL/dsigma of this step (last step), or nullptr
    double* part_sig;       // [SG][NS][Npad] k_adj_sig: partial sums of the forward integrand per chunk group
    double* lt;             // [DD][Npad] pairing matrix of lambda(sigma_struc) / G_inf-scaled (k_adj_node)
    double* part_adj;       // [SG][DD + 2][Npad] k_adj_hist: partial lambda(A), lambda(1/tau), lambda(1/gamma_c)
    long long t_off;        // step t = *t0 + t_off (the segment's first step lives in device memory, so that
    const long long* t0;    // one captured graph serves every segment)
    int B, C, S;            // history grid; S slot chunks of the split kernels
    int cpb, SG;            // chunks per block of the split kernels (a power of two <= 16) and chunk groups
};

// Thread -> (node, chunk) of the split kernels: a block of 128 threads holds G = 128 / cpb nodes x cpb
// chunks, consecutive threads on consecutive nodes of one chunk; block b covers node group b % (Npad / G)
// and chunk group b / (Npad / G).  The block adds its cpb chunks of every node itself (chunk_group_sum), so
// that the per-node FP64 kernels add SG = S / cpb group sums instead of S chunk sums.
struct SplitIdx { int n, chunk, nl, cl, G, group; };
__device__ inline SplitIdx split_idx(int cpb, long long Npad) {
    SplitIdx x;
    x.G = blockDim.x / cpb;
    x.nl = threadIdx.x % x.G;
    x.cl = threadIdx.x / x.G;
    const int ngroups = (int)(Npad / x.G);
    x.group = blockIdx.x / ngroups;
    x.n = (blockIdx.x % ngroups) * x.G + x.nl;
    x.chunk = x.group * cpb + x.cl;
    return x;
}

// Sum of the M values v of the block's cpb chunks of each node, by a fixed pairwise tree in shared memory
// (s_red: blockDim.x * M doubles); every thread of the block calls it; the sums are valid in the threads of
// chunk cl = 0 (returned in v).
template <int M>
__device__ inline void chunk_group_sum(double* s_red, const SplitIdx& x, int cpb, double* v) {
#pragma unroll
    for (int i = 0; i < M; ++i) s_red[threadIdx.x * M + i] = v[i];
    __syncthreads();
    for (int st = cpb / 2; st >= 1; st /= 2) {
        if (x.cl < st)
#pragma unroll
            for (int i = 0; i < M; ++i) s_red[threadIdx.x * M + i] += s_red[(threadIdx.x + st * x.G) * M + i];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = s_red[threadIdx.x * M + i];
}

// Slot range [l0, l1) of chunk `chunk` of S over Ls slots.
__device__ inline void adj_chunk(int Ls, int S, int chunk, int* l0, int* l1) {
    const int len = (Ls + S - 1) / S;
    *l0 = min(Ls, chunk * len);
    *l1 = min(Ls, *l0 + len);
}

// The per-CTA table of slot roles at step t (ages, weights, merge partners; same as the sweep's).
template <class A>
__device__ inline long long adj_t(const A& a) { return *a.t0 + a.t_off; }

template <class A>
__device__ inline void adj_table(const A& a, float* s_age, float* s_w, int* s_part, BlockStep* s_bs) {
    const int Ls = a.B * a.C;
    sched_step_cta(a.B, a.C, adj_t(a), s_bs);
    __syncthreads();
    for (int l = threadIdx.x; l < Ls; l += blockDim.x) {
        int age, part;
        const float w = sched_slot_role(s_bs, a.C, l / a.C, l % a.C, &age, &part);
        s_age[l] = (float)age;
        s_w[l] = w;
        s_part[l] = part;
    }
    __syncthreads();
}

// Forward recompute of the history sweep of step t on the taped history: per (node, chunk) thread the
// partial sum of the integrand over the chunk's slots (point_update on a copy; the tape is read only).
template <int D, typename TP, typename TH>
__global__ void __launch_bounds__(128) k_adj_sig(AdjArgs<TP, TH> a, Geom g, AdjPar p) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    const int Ls = a.B * a.C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_age = reinterpret_cast<float*>(smem_raw);
    float* s_w = s_age + Ls;
    int* s_part = reinterpret_cast<int*>(s_w + Ls);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(s_part + Ls);
    adj_table(a, s_age, s_w, s_part, s_bs);
    __shared__ double s_red[128 * NS];
    const SplitIdx x = split_idx(a.cpb, g.Npad);
    const int n = x.n, chunk = x.chunk;
    const bool active = chunk < a.S && n < g.N;
    const long long Np = g.Npad;
    using R = TH;   // the forward sweep's arithmetic
    const long long s_last = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_prev;
    R kl[DD], A[DD];
    for (int c = 0; c < DD; ++c) kl[c] = active ? a.K[(s_last * DD + c) * Np + n] : R(0);
    expm1_mat<D, R>(kl, A);
    R acc[NS];
    for (int i = 0; i < NS; ++i) acc[i] = 0;
    int l0 = 0, l1 = 0;
    if (active) adj_chunk(Ls, a.S, chunk, &l0, &l1);
    for (int l = l0; l < l1; ++l) {
        const float w = s_w[l];
        if (w == 0.0f) continue;
        R Xl[DD], kap[DD];
        for (int c = 0; c < DD; ++c) {
            Xl[c] = a.X[((long long)l * DD + c) * Np + n];
            kap[c] = a.K[((long long)l * DD + c) * Np + n];
        }
        const int part = s_part[l];
        if (part >= 0)
            for (int c = 0; c < DD; ++c) kap[c] = R(0.5) * (kap[c] + a.K[((long long)part * DD + c) * Np + n]);
        point_update<D, R>(Xl, A, kap, (R)s_age[l], (R)w, (R)p.inv_tau, (R)p.inv_gc, acc);
    }
    double v[NS];
    for (int i = 0; i < NS; ++i) v[i] = (double)acc[i];
    chunk_group_sum<NS>(s_red, x, a.cpb, v);
    if (x.cl == 0 && n < g.N)
        for (int i = 0; i < NS; ++i) a.part_sig[((long long)x.group * NS + i) * Np + n] = v[i];
}

template <int Q, typename TP, typename TH>
__global__ void __launch_bounds__(32) k_adj_node(AdjArgs<TP, TH> a, Geom g, AdjPar p) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    // only the block transitions of step t are needed here (the merges of the commit)
    __shared__ BlockStep s_bs[LBVE_MAXB];
    sched_step_cta(a.B, a.C, adj_t(a), s_bs);
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    const long long Np = g.Npad;
    const Chan& ch = g.ch[0];

    // ---------------- forward recompute of step t at this node ----------------
    double dn[Q], dr = 0.0, J[3] = {0, 0, 0};
    for (int q = 0; q < Q; ++q) {
        dn[q] = a.n[q * Np + n];
        dr += dn[q];
        J[0] += L::cx(q) * dn[q];
        J[1] += L::cy(q) * dn[q];
        if (D == 3) J[2] += L::cz(q) * dn[q];
    }
    double kt[DD];
    kappa_fd<D>(a.u_raw, Np, ch, n, kt);
    double acc[NS];   // the history sum of step t (k_adj_sig's chunks, in chunk order)
    for (int i = 0; i < NS; ++i) acc[i] = 0.0;
#pragma unroll 16   // the groups' loads in flight together (the additions keep their order)
    for (int c = 0; c < a.SG; ++c)
#pragma unroll
        for (int i = 0; i < NS; ++i) acc[i] += a.part_sig[((long long)c * NS + i) * Np + n];
    double newp[NS];   // the point created now: (kappa + kappa^T)/2 packed
    if (D == 2) {
        newp[0] = kt[0]; newp[1] = kt[3]; newp[2] = 0.5 * (kt[1] + kt[2]);
    } else {
        newp[0] = kt[0]; newp[1] = kt[4]; newp[2] = kt[8];
        newp[3] = 0.5 * (kt[1] + kt[3]); newp[4] = 0.5 * (kt[2] + kt[6]); newp[5] = 0.5 * (kt[5] + kt[7]);
    }
    double sg[NS];
    for (int i = 0; i < NS; ++i) sg[i] = p.G_inf * (acc[i] + newp[i]);
    // collision quantities
    double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (D == 2) {
        S[0][0] = sg[0]; S[1][1] = sg[1]; S[0][1] = S[1][0] = sg[2];
    } else {
        S[0][0] = sg[0]; S[1][1] = sg[1]; S[2][2] = sg[2];
        S[0][1] = S[1][0] = sg[3]; S[0][2] = S[2][0] = sg[4]; S[1][2] = S[2][1] = sg[5];
    }
    double tr = 0.0;
    for (int c = 0; c < D; ++c) tr += S[c][c];
    const double ddr = p.trace_full ? -(tr - a.trp[n]) * (3.0 / D) : 0.0;
    const double drho = dr + 0.5 * ddr;
    const double rho = p.rho0 + drho;
    double u[3] = {0, 0, 0};
    for (int c = 0; c < D; ++c) u[c] = (J[c] + 0.5 * p.f[c]) / rho;
    double uu = 0.0;
    for (int c = 0; c < D; ++c) uu += u[c] * u[c];
    const double omega = 1.0 / p.tau_lb, fpre = 1.0 - 0.5 * omega, cs2 = 1.0 / 3.0;

    // ---------------- adjoint of collision and streaming ----------------
    double lam_dr = 0.0, lam_J[3] = {0, 0, 0}, lam_f[3] = {0, 0, 0}, lam_u[3] = {0, 0, 0};
    double lam_rho = 0.0, lam_drho = 0.0, lam_ddr = 0.0, lam_uu = 0.0, lam_trX = 0.0;
    double lam_Sb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, lam_Xf[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    int x, y, z;
    node_xyz(ch, n, x, y, z);
    for (int q = 0; q < Q; ++q) {
        const int cq[3] = {L::cx(q), L::cy(q), L::cz(q)};
        // lambda of this population after streaming (push adjoint = pull)
        int xd = x + cq[0];
        xd = xd < 0 ? ch.nx - 1 : (xd >= ch.nx ? 0 : xd);
        const int yd = y + cq[1];
        bool wall = yd < 0 || yd >= ch.ny;
        int zd = z + cq[2];
        if (D == 3) {
            if (ch.wall_z) wall = wall || zd < 0 || zd >= ch.nz;
            else zd = zd < 0 ? ch.nz - 1 : (zd >= ch.nz ? 0 : zd);
        }
        const double lpost = wall ? a.lam_n1[L::opp(q) * Np + n] : a.lam_n1[q * Np + (xd + ch.nx * (yd + ch.ny * zd))];
        // post = (1 - omega) n + omega dneq + F
        a.lam_n0[q * Np + n] = (1.0 - omega) * lpost;
        const double wq = L::w(q);
        double cu = 0.0, cf = 0.0;
        for (int r = 0; r < D; ++r) { cu += cq[r] * u[r]; cf += cq[r] * p.f[r]; }
        const double l_dneq = omega * lpost, l_F = lpost;
        // dneq = w (drho + rho (3 cu + 4.5 cu^2 - 1.5 uu))
        lam_drho += wq * l_dneq;
        lam_rho += wq * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu) * l_dneq;
        const double l_cu = wq * rho * (3.0 + 9.0 * cu) * l_dneq;
        lam_uu += wq * rho * (-1.5) * l_dneq;
        // F = w (-4.5 omega cSc + fpre (ddr + 3 cf + 4.5 cXc - 4.5 cs2 trX))
        const double l_cSc = -4.5 * omega * wq * l_F;
        lam_ddr += fpre * wq * l_F;
        const double l_cf = 3.0 * fpre * wq * l_F;
        const double l_cXc = 4.5 * fpre * wq * l_F;
        lam_trX += -4.5 * cs2 * fpre * wq * l_F;
        for (int r = 0; r < D; ++r) {
            lam_u[r] += cq[r] * l_cu;
            lam_f[r] += cq[r] * l_cf;
            for (int c = 0; c < D; ++c) {
                lam_Sb[r][c] += cq[r] * cq[c] * l_cSc;
                lam_Xf[r][c] += cq[r] * cq[c] * l_cXc;
            }
        }
    }
    for (int c = 0; c < D; ++c) lam_Xf[c][c] += lam_trX;
    // Xf_ab = -ddr u_a u_b + u_b f_a + u_a f_b
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            const double l = lam_Xf[r][c];
            lam_ddr += -u[r] * u[c] * l;
            lam_u[r] += (-ddr * u[c] + p.f[c]) * l;
            lam_u[c] += (-ddr * u[r] + p.f[r]) * l;
            lam_f[r] += u[c] * l;
            lam_f[c] += u[r] * l;
        }
    for (int c = 0; c < D; ++c) lam_u[c] += 2.0 * u[c] * lam_uu;
    if (a.seed_u)
        for (int c = 0; c < D; ++c) lam_u[c] += a.seed_u[c * Np + n];
    // u = (J + f/2) / rho
    for (int c = 0; c < D; ++c) {
        lam_J[c] += lam_u[c] / rho;
        lam_f[c] += 0.5 * lam_u[c] / rho;
        lam_rho += -u[c] * lam_u[c] / rho;
    }
    lam_drho += lam_rho;
    lam_dr += lam_drho;
    lam_ddr += 0.5 * lam_drho;
    // S_bar = sigma - tr/D; ddr = -(tr - trp) 3/D; the next step's tr_prev = tr
    double lam_tr = a.lam_trp[n];
    if (p.trace_full) {
        lam_tr += -(3.0 / D) * lam_ddr;
        a.lam_trp[n] = (3.0 / D) * lam_ddr;
    } else {
        a.lam_trp[n] = 0.0;
    }
    double lam_sg[NS];
    for (int c = 0; c < D; ++c) lam_tr += -lam_Sb[c][c] / D;
    if (D == 2) {
        lam_sg[0] = lam_Sb[0][0] + lam_tr; lam_sg[1] = lam_Sb[1][1] + lam_tr; lam_sg[2] = lam_Sb[0][1] + lam_Sb[1][0];
    } else {
        lam_sg[0] = lam_Sb[0][0] + lam_tr; lam_sg[1] = lam_Sb[1][1] + lam_tr; lam_sg[2] = lam_Sb[2][2] + lam_tr;
        lam_sg[3] = lam_Sb[0][1] + lam_Sb[1][0]; lam_sg[4] = lam_Sb[0][2] + lam_Sb[2][0];
        lam_sg[5] = lam_Sb[1][2] + lam_Sb[2][1];
    }
    if (a.seed_s)
        for (int i = 0; i < NS; ++i) lam_sg[i] += a.seed_s[i * Np + n];

    // ---------------- adjoint of the commit ----------------
    double lam_G = 0.0, lam_acc[NS], lam_kt[DD];
    for (int i = 0; i < NS; ++i) {
        lam_G += (acc[i] + newp[i]) * lam_sg[i];
        lam_acc[i] = p.G_inf * lam_sg[i];
    }
    for (int c = 0; c < DD; ++c) lam_kt[c] = 0.0;
    if (D == 2) {
        lam_kt[0] += lam_acc[0]; lam_kt[3] += lam_acc[1];
        lam_kt[1] += 0.5 * lam_acc[2]; lam_kt[2] += 0.5 * lam_acc[2];
    } else {
        lam_kt[0] += lam_acc[0]; lam_kt[4] += lam_acc[1]; lam_kt[8] += lam_acc[2];
        lam_kt[1] += 0.5 * lam_acc[3]; lam_kt[3] += 0.5 * lam_acc[3];
        lam_kt[2] += 0.5 * lam_acc[4]; lam_kt[6] += 0.5 * lam_acc[4];
        lam_kt[5] += 0.5 * lam_acc[5]; lam_kt[7] += 0.5 * lam_acc[5];
    }
    // new point (last forward operation): X_dst = 0, K_dst = kappa(t)
    {
        const long long dst = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
        for (int c = 0; c < DD; ++c) {
            lam_kt[c] += (double)a.lamK[(dst * DD + c) * Np + n];
            a.lamK[(dst * DD + c) * Np + n] = TH(0);
            a.lamX[(dst * DD + c) * Np + n] = TH(0);
        }
    }
    // merges in reverse order (finest first): X_dst = X'_o1, K_dst = (K_o1 + K_o2)/2
    for (int bb = a.B - 1; bb >= 1; --bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long src1 = (long long)bb * a.C + o1, src2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
        for (int c = 0; c < DD; ++c) {
            const double lx = a.lamX[(dst * DD + c) * Np + n], lk = a.lamK[(dst * DD + c) * Np + n];
            a.lamX[(dst * DD + c) * Np + n] = TH(0);
            a.lamK[(dst * DD + c) * Np + n] = TH(0);
            a.lamX[(src1 * DD + c) * Np + n] = (TH)((double)a.lamX[(src1 * DD + c) * Np + n] + lx);
            a.lamK[(src1 * DD + c) * Np + n] = (TH)((double)a.lamK[(src1 * DD + c) * Np + n] + 0.5 * lk);
            a.lamK[(src2 * DD + c) * Np + n] = (TH)((double)a.lamK[(src2 * DD + c) * Np + n] + 0.5 * lk);
        }
    }

    // ---------------- pairing matrix for the adjoint of the history sweep (k_adj_hist) ----------------
    {
        double Lt[DD];
        packed_to_pairing<D>(lam_acc, Lt);
        for (int c = 0; c < DD; ++c) a.lt[c * Np + n] = Lt[c];
    }

    // ---------------- outputs ----------------
    for (int c = 0; c < DD; ++c) a.lam_kt[c * Np + n] = lam_kt[c];
    for (int q = 0; q < Q; ++q) {
        double l = lam_dr;
        l += L::cx(q) * lam_J[0] + L::cy(q) * lam_J[1];
        if (D == 3) l += L::cz(q) * lam_J[2];
        a.lam_n0[q * Np + n] += l;
    }
    a.lam_theta[0 * Np + n] += lam_G;
    a.lam_theta[3 * Np + n] += p.rho0 * lam_f[0];                                // f_x = rho0 g_x
}

// Adjoint of the history sweep of step t, per (node, chunk) thread over the chunk's slots: lambda of each
// point's X and kappa (in place; the newer half of a merge has weight 0 and is not visited, so every lamK
// entry has a single writer), and the chunk's partial lambda(A), lambda(1/tau), lambda(1/gamma_c).
template <int D, typename TP, typename TH>
__global__ void __launch_bounds__(128) k_adj_hist(AdjArgs<TP, TH> a, Geom g, AdjPar p) {
    constexpr int DD = D * D;
    const int Ls = a.B * a.C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_age = reinterpret_cast<float*>(smem_raw);
    float* s_w = s_age + Ls;
    int* s_part = reinterpret_cast<int*>(s_w + Ls);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(s_part + Ls);
    adj_table(a, s_age, s_w, s_part, s_bs);
    __shared__ double s_red[128 * (DD + 2)];
    const SplitIdx x = split_idx(a.cpb, g.Npad);
    const int n = x.n, chunk = x.chunk;
    const bool active = chunk < a.S && n < g.N;
    const long long Np = g.Npad;
    using R = TH;   // the forward sweep's arithmetic; the chunk's rate parts in double
    const long long s_last = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_prev;
    R kl[DD], A[DD], Lt[DD], lamA[DD];
    for (int c = 0; c < DD; ++c) {
        kl[c] = active ? a.K[(s_last * DD + c) * Np + n] : R(0);
        Lt[c] = active ? (R)a.lt[c * Np + n] : R(0);
        lamA[c] = 0;
    }
    expm1_mat<D, R>(kl, A);
    double lam_it = 0.0, lam_ig = 0.0;
    int l0 = 0, l1 = 0;
    if (active) adj_chunk(Ls, a.S, chunk, &l0, &l1);
    for (int l = l0; l < l1; ++l) {
        const float w = s_w[l];
        if (w == 0.0f) continue;
        R Xl[DD], Xn[DD], kap[DD], lX[DD], lk[DD];
        for (int c = 0; c < DD; ++c) {
            Xl[c] = a.X[((long long)l * DD + c) * Np + n];
            kap[c] = a.K[((long long)l * DD + c) * Np + n];
            lX[c] = a.lamX[((long long)l * DD + c) * Np + n];   // lambda of X' (after the sweep)
            lk[c] = 0;
        }
        const int part = s_part[l];
        if (part >= 0)
            for (int c = 0; c < DD; ++c) kap[c] = R(0.5) * (kap[c] + a.K[((long long)part * DD + c) * Np + n]);
        // X' = X + A + A X
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) {
                R s = Xl[r * D + c] + A[r * D + c];
                for (int k = 0; k < D; ++k) s += A[r * D + k] * Xl[k * D + c];
                Xn[r * D + c] = s;
            }
        integrand_adjoint<D, R>(Xn, kap, (R)s_age[l], (R)w, (R)p.inv_tau, (R)p.inv_gc, Lt, lX, lk, &lam_it, &lam_ig);
        // lambda A += lX (1 + X)^T ; lambda X = (1 + A)^T lX
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) {
                R s = lX[r * D + c];
                for (int k = 0; k < D; ++k) s += lX[r * D + k] * Xl[c * D + k];
                lamA[r * D + c] += s;
            }
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) {
                R s = lX[r * D + c];
                for (int k = 0; k < D; ++k) s += A[k * D + r] * lX[k * D + c];
                Xn[r * D + c] = s;   // reuse as lambda X (before the sweep)
            }
        for (int c = 0; c < DD; ++c) a.lamX[((long long)l * DD + c) * Np + n] = Xn[c];
        if (part >= 0) {
            for (int c = 0; c < DD; ++c) {
                a.lamK[((long long)l * DD + c) * Np + n] += R(0.5) * lk[c];
                a.lamK[((long long)part * DD + c) * Np + n] += R(0.5) * lk[c];
            }
        } else {
            for (int c = 0; c < DD; ++c) a.lamK[((long long)l * DD + c) * Np + n] += lk[c];
        }
    }
    double v[DD + 2];
    for (int c = 0; c < DD; ++c) v[c] = (double)lamA[c];
    v[DD] = lam_it;
    v[DD + 1] = lam_ig;
    chunk_group_sum<DD + 2>(s_red, x, a.cpb, v);
    if (x.cl == 0 && n < g.N) {
        double* out = a.part_adj + (long long)x.group * (DD + 2) * Np + n;
        for (int c = 0; c < DD + 2; ++c) out[c * Np] = v[c];
    }
}

// The chunk sums of k_adj_hist (chunk order), the adjoint of A = exp(kappa(t-1)) - 1 (kappa(t-1) is the kappa
// of the newest stored point) and the rate parts of dL/dtheta.
template <int D, typename TP, typename TH>
__global__ void __launch_bounds__(32) k_adj_fin(AdjArgs<TP, TH> a, Geom g, AdjPar p) {
    constexpr int DD = D * D;
    __shared__ BlockStep bs[LBVE_MAXB];
    sched_step_cta(a.B, a.C, adj_t(a), bs);
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    const long long Np = g.Npad;
    double lamA[DD], lam_it = 0.0, lam_ig = 0.0;
    for (int c = 0; c < DD; ++c) lamA[c] = 0.0;
#pragma unroll 16   // the groups' loads in flight together (the additions keep their order)
    for (int ch = 0; ch < a.SG; ++ch) {
        const double* in = a.part_adj + (long long)ch * (DD + 2) * Np + n;
        for (int c = 0; c < DD; ++c) lamA[c] += in[c * Np];
        lam_it += in[DD * Np];
        lam_ig += in[(DD + 1) * Np];
    }
    const long long s_last = (long long)(a.B - 1) * a.C + bs[a.B - 1].head_prev;
    double kl[DD], lk[DD];
    for (int c = 0; c < DD; ++c) {
        kl[c] = a.K[(s_last * DD + c) * Np + n];
        lk[c] = 0.0;
    }
    expm1_adjoint<D, sizeof(TH) == 4 ? 4 : 8>(kl, lamA, lk);   // the order the forward's history type used
    for (int c = 0; c < DD; ++c) a.lamK[(s_last * DD + c) * Np + n] = (TH)((double)a.lamK[(s_last * DD + c) * Np + n] + lk[c]);
    a.lam_theta[1 * Np + n] += lam_it * (-1.0 / (p.tau * p.tau));                // d(1/tau)/dtau
    a.lam_theta[2 * Np + n] += isinf(p.gamma_c) ? 0.0 : lam_ig * (-1.0 / (p.gamma_c * p.gamma_c));
}

// Forward weight of node yn in the finite-difference stencil of node xn along `axis` (Sec. III:
// central; at a wall-adjacent node the three-point formula through the wall).
__device__ inline double fd_weight(const Chan& c, int axis, int xn, int yn) {
    int x, y, z;
    node_xyz(c, xn, x, y, z);
    const int i = axis == 0 ? x : (axis == 1 ? y : z);
    const int nn = axis == 0 ? c.nx : (axis == 1 ? c.ny : c.nz);
    const bool periodic = axis == 0 || (axis == 2 && !c.wall_z);
    auto node_at = [&](int j) {
        int xx = x, yy = y, zz = z;
        if (axis == 0) xx = j; else if (axis == 1) yy = j; else zz = j;
        return c.off + xx + c.nx * (yy + c.ny * zz);
    };
    double w = 0.0;
    if (periodic) {
        const int jp = (i + 1) % nn, jm = (i - 1 + nn) % nn;
        if (node_at(jp) == yn) w += 0.5;
        if (node_at(jm) == yn) w -= 0.5;
        return w;
    }
    if (i == 0) {
        if (node_at(0) == yn) w += 1.0;
        if (nn > 1 && node_at(1) == yn) w += 1.0 / 3.0;
        return w;
    }
    if (i == nn - 1) {
        if (node_at(nn - 1) == yn) w -= 1.0;
        if (node_at(nn - 2) == yn) w -= 1.0 / 3.0;
        return w;
    }
    if (node_at(i + 1) == yn) w += 0.5;
    if (node_at(i - 1) == yn) w -= 0.5;
    return w;
}

// Transpose of the finite differences and adjoint of the raw moments at node n.
template <int Q, typename TP>
__global__ void __launch_bounds__(128) k_adj_fd(const TP* __restrict__ pops, const double* __restrict__ lam_kt,
                                                double* __restrict__ lam_n0, double* __restrict__ lam_theta, Geom g,
                                                AdjPar p) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    constexpr int DD = D * D;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    const long long Np = g.Npad;
    const Chan& ch = g.ch[0];
    int x, y, z;
    node_xyz(ch, n, x, y, z);
    // lambda u_raw(n) = sum over stencils that read n
    double lam_ur[3] = {0, 0, 0};
    for (int axis = 0; axis < D; ++axis) {
        const int nn = axis == 0 ? ch.nx : (axis == 1 ? ch.ny : ch.nz);
        const int i = axis == 0 ? x : (axis == 1 ? y : z);
        int cand[3];
        int nc = 0;
        for (int dlt = -1; dlt <= 1; ++dlt) {
            int j = i + dlt;
            const bool periodic = axis == 0 || (axis == 2 && !ch.wall_z);
            if (periodic) j = (j + nn) % nn;
            else if (j < 0 || j >= nn) continue;
            int xx = x, yy = y, zz = z;
            if (axis == 0) xx = j; else if (axis == 1) yy = j; else zz = j;
            const int m = ch.off + xx + ch.nx * (yy + ch.ny * zz);
            bool seen = false;
            for (int k = 0; k < nc; ++k) seen = seen || cand[k] == m;
            if (!seen) cand[nc++] = m;
        }
        for (int k = 0; k < nc; ++k) {
            const double wgt = fd_weight(ch, axis, cand[k], n);
            if (wgt == 0.0) continue;
            for (int a = 0; a < D; ++a) lam_ur[a] += wgt * lam_kt[(a * D + axis) * Np + cand[k]];
        }
    }
    // u_raw = (J + f/2) / (rho0 + dr)
    double dr = 0.0, J[3] = {0, 0, 0};
    for (int q = 0; q < Q; ++q) {
        const double v = (double)pops[q * Np + n];
        dr += v;
        J[0] += L::cx(q) * v;
        J[1] += L::cy(q) * v;
        if (D == 3) J[2] += L::cz(q) * v;
    }
    const double rr = p.rho0 + dr;
    double lam_dr = 0.0, lam_J[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
        const double ur = (J[a] + 0.5 * p.f[a]) / rr;
        lam_J[a] += lam_ur[a] / rr;
        lam_dr += -ur * lam_ur[a] / rr;
        if (a == 0) lam_theta[3 * Np + n] += p.rho0 * 0.5 * lam_ur[0] / rr;
    }
    for (int q = 0; q < Q; ++q) {
        double l = lam_dr + L::cx(q) * lam_J[0] + L::cy(q) * lam_J[1];
        if (D == 3) l += L::cz(q) * lam_J[2];
        lam_n0[q * Np + n] += l;
    }
    (void)DD;
}

}  // namespace lbk
