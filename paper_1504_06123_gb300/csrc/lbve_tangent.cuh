// lbve_tangent.cuh -- tangent-linear (forward-mode) model of the hybrid step: every state value carries
// its derivatives with respect to the four model parameters theta = (G_inf, tau, gamma_c, g_x).
//
// The differentiated step is the same method as the plain kernels (Sec. III; Eqs. gitt, nlmax, eeval,
// bodyforce, hydrofields): moments, kappa by finite differences, history (advance E, trapezoidal sum,
// merges, new point), trace split, density source, BGK collision with forcing, streaming.  It runs in
// double precision on one channel, one thread per node (the differentiation workloads are small:
// hundreds of nodes).  Derivatives of the parameters themselves: dG_inf/dtheta_0 = 1,
// d(1/tau)/dtheta_1 = -1/tau^2, d(1/gamma_c)/dtheta_2 = -1/gamma_c^2, d(rho0 g_x)/dtheta_3 = rho0.
// At gammadot = 0 the derivative of sqrt is taken as 0 (the subgradient of |gammadot|).
#pragma once
#include "lbve_kernels.cuh"

namespace lbk {

constexpr int NT = 4;   // tangent directions

struct Dual {
    double v;
    double d[NT];
    Dual() = default;
    __host__ __device__ Dual(double x) : v(x), d{0.0, 0.0, 0.0, 0.0} {}
};

__host__ __device__ inline Dual operator+(const Dual& a, const Dual& b) {
    Dual r; r.v = a.v + b.v;
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
__host__ __device__ inline Dual operator-(const Dual& a, const Dual& b) {
    Dual r; r.v = a.v - b.v;
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
__host__ __device__ inline Dual operator-(const Dual& a) {
    Dual r; r.v = -a.v;
    for (int i = 0; i < NT; ++i) r.d[i] = -a.d[i];
    return r;
}
__host__ __device__ inline Dual operator*(const Dual& a, const Dual& b) {
    Dual r; r.v = a.v * b.v;
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
__host__ __device__ inline Dual operator/(const Dual& a, const Dual& b) {
    Dual r; r.v = a.v / b.v;
    const double ib = 1.0 / b.v;
    for (int i = 0; i < NT; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
__host__ __device__ inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
__host__ __device__ inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
__host__ __device__ inline Dual operator*(double a, const Dual& b) { return Dual(a) * b; }
__host__ __device__ inline Dual operator*(int a, const Dual& b) { return Dual((double)a) * b; }

__device__ inline Dual exp(const Dual& a) {
    const double e = ::exp(a.v);
    Dual r; r.v = e;
    for (int i = 0; i < NT; ++i) r.d[i] = e * a.d[i];
    return r;
}
__device__ inline Dual sqrt(const Dual& a) {
    const double s = ::sqrt(a.v);
    Dual r; r.v = s;
    for (int i = 0; i < NT; ++i) r.d[i] = s > 0.0 ? a.d[i] / (2.0 * s) : 0.0;
    return r;
}

template <> struct FastMath<Dual> {
    __device__ static __forceinline__ Dual exp_neg(const Dual& x) { return exp(-x); }
    __device__ static __forceinline__ Dual sqrt_pos(const Dual& x) { return sqrt(x); }
};

// The parameters as duals (value and derivative with respect to theta).
struct TanPar {
    Dual G_inf, inv_tau, inv_gc, f[3];
    double rho0, tau_lb;
    int trace_full;
};

// Moments and advance of the step counter.
template <int Q>
__global__ void __launch_bounds__(128) k_moments_t(const Dual* __restrict__ dn, Dual* __restrict__ u_raw, Geom g,
                                                   TanPar p, long long* t_dev) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) *t_dev += 1;
    if (n >= g.N) return;
    Dual drho(0.0), j[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const Dual v = dn[(long long)q * g.Npad + n];
        drho += v;
        if (L::cx(q)) j[0] += L::cx(q) * v;
        if (L::cy(q)) j[1] += L::cy(q) * v;
        if (D == 3 && L::cz(q)) j[2] += L::cz(q) * v;
    }
    const Dual inv = Dual(1.0) / (Dual(p.rho0) + drho);
#pragma unroll
    for (int a = 0; a < D; ++a) u_raw[(long long)a * g.Npad + n] = (j[a] + 0.5 * p.f[a]) * inv;
}

// The per-CTA table of slot roles at step t (ages, weights, merge partners).
__device__ inline void tan_table(int B, int C, long long t, float* s_age, float* s_w, int* s_part, BlockStep* s_bs) {
    const int L = B * C;
    sched_step_cta(B, C, t, s_bs);
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int age, part;
        const float w = sched_slot_role(s_bs, C, l / C, l % C, &age, &part);
        s_age[l] = (float)age;
        s_w[l] = w;
        s_part[l] = part;
    }
    __syncthreads();
}

// History sweep in duals, one thread per (node, slot chunk): advance E - 1 in place over the chunk's slots
// and write the chunk's partial trapezoidal sum (added in chunk order by k_history_t).
template <int D>
__global__ void __launch_bounds__(128) k_sweep_t(Dual* __restrict__ X, const Dual* __restrict__ K,
                                                 Dual* __restrict__ part_t, Geom g, TanPar p,
                                                 const long long* t_dev, int B, int C, int S) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    const int L = B * C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_age = reinterpret_cast<float*>(smem_raw);
    float* s_w = s_age + L;
    int* s_part = reinterpret_cast<int*>(s_w + L);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(s_part + L);
    tan_table(B, C, *t_dev, s_age, s_w, s_part, s_bs);
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int n = (int)(idx % g.Npad), chunk = (int)(idx / g.Npad);
    if (chunk >= S || n >= g.N) return;
    const long long Np = g.Npad;
    Dual A[DD];
    {
        const long long s_last = (long long)(B - 1) * C + s_bs[B - 1].head_prev;
        Dual kp[DD];
        for (int c = 0; c < DD; ++c) kp[c] = K[(s_last * DD + c) * Np + n];
        expm1_mat<D>(kp, A);
    }
    Dual acc[NS];
    for (int i = 0; i < NS; ++i) acc[i] = Dual(0.0);
    const int len = (L + S - 1) / S;
    const int l0 = min(L, chunk * len), l1 = min(L, l0 + len);
    for (int l = l0; l < l1; ++l) {
        const float w = s_w[l];
        if (w == 0.0f) continue;
        Dual Xl[DD], kap[DD];
        for (int c = 0; c < DD; ++c) {
            Xl[c] = X[((long long)l * DD + c) * Np + n];
            kap[c] = K[((long long)l * DD + c) * Np + n];
        }
        const int part = s_part[l];
        if (part >= 0)
            for (int c = 0; c < DD; ++c) kap[c] = 0.5 * (kap[c] + K[((long long)part * DD + c) * Np + n]);
        point_update<D>(Xl, A, kap, Dual((double)s_age[l]), Dual((double)w), p.inv_tau, p.inv_gc, acc);
        for (int c = 0; c < DD; ++c) X[((long long)l * DD + c) * Np + n] = Xl[c];
    }
    for (int i = 0; i < NS; ++i) part_t[((long long)chunk * NS + i) * Np + n] = acc[i];
}

// The node's history commit in duals after k_sweep_t: the chunk sums plus the point created now give
// sigma_struc(t); then the merges and the new point (form "P": E - 1 advanced in place).
template <int D>
__global__ void __launch_bounds__(128) k_history_t(Dual* __restrict__ X, Dual* __restrict__ K,
                                                   const Dual* __restrict__ u_raw, Dual* __restrict__ kappa_f,
                                                   Dual* __restrict__ sigma_f, const Dual* __restrict__ part_t,
                                                   Geom g, TanPar p, const long long* t_dev, int B, int C, int S) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_age = reinterpret_cast<float*>(smem_raw);
    float* s_w = s_age + B * C;
    int* s_part = reinterpret_cast<int*>(s_w + B * C);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(s_part + B * C);
    tan_table(B, C, *t_dev, s_age, s_w, s_part, s_bs);
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    const long long Np = g.Npad;
    Dual acc[NS];
    for (int i = 0; i < NS; ++i) acc[i] = Dual(0.0);
    for (int c = 0; c < S; ++c)
        for (int i = 0; i < NS; ++i) acc[i] += part_t[((long long)c * NS + i) * Np + n];
    Dual kt[DD];
    kappa_fd<D>(u_raw, Np, g.ch[0], n, kt);
    if (D == 2) {
        acc[0] += 0.5 * (kt[0] + kt[0]);
        acc[1] += 0.5 * (kt[3] + kt[3]);
        acc[2] += 0.5 * (kt[1] + kt[2]);
    } else {
        acc[0] += 0.5 * (kt[0] + kt[0]);
        acc[1] += 0.5 * (kt[4] + kt[4]);
        acc[2] += 0.5 * (kt[8] + kt[8]);
        acc[3] += 0.5 * (kt[1] + kt[3]);
        acc[4] += 0.5 * (kt[2] + kt[6]);
        acc[5] += 0.5 * (kt[5] + kt[7]);
    }
    for (int i = 0; i < NS; ++i) sigma_f[i * Np + n] = p.G_inf * acc[i];
    for (int c = 0; c < DD; ++c) kappa_f[c * Np + n] = kt[c];
    for (int bb = 1; bb < B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (C - 1); if (o1 < 0) o1 += C;
        int o2 = b.head_prev - (C - 2); if (o2 < 0) o2 += C;
        const long long src1 = (long long)bb * C + o1, src2 = (long long)bb * C + o2;
        const long long dst = (long long)(bb - 1) * C + s_bs[bb - 1].head_new;
        for (int c = 0; c < DD; ++c) {
            X[(dst * DD + c) * Np + n] = X[(src1 * DD + c) * Np + n];
            K[(dst * DD + c) * Np + n] = 0.5 * (K[(src1 * DD + c) * Np + n] + K[(src2 * DD + c) * Np + n]);
        }
    }
    const long long dst = (long long)(B - 1) * C + s_bs[B - 1].head_new;
    for (int c = 0; c < DD; ++c) {
        X[(dst * DD + c) * Np + n] = Dual(0.0);
        K[(dst * DD + c) * Np + n] = kt[c];
    }
}

// Collision with the forcing of Eq. (bodyforce) and push streaming, in duals.
template <int Q>
__global__ void __launch_bounds__(128) k_collide_t(const Dual* __restrict__ dn_in, Dual* __restrict__ dn_out,
                                                   const Dual* __restrict__ sigma, Dual* __restrict__ tr_prev,
                                                   Dual* __restrict__ rho_f, Dual* __restrict__ u_f, Geom g, TanPar p) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    const long long Np = g.Npad;
    const Chan& ch = g.ch[0];
    const double cs2 = 1.0 / 3.0;
    Dual dn[Q];
    Dual drho_raw(0.0), j[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        dn[q] = dn_in[q * Np + n];
        drho_raw += dn[q];
        if (L::cx(q)) j[0] += L::cx(q) * dn[q];
        if (L::cy(q)) j[1] += L::cy(q) * dn[q];
        if (D == 3 && L::cz(q)) j[2] += L::cz(q) * dn[q];
    }
    Dual S[3][3];
    Dual tr(0.0);
    if (D == 2) {
        S[0][0] = sigma[0 * Np + n]; S[1][1] = sigma[1 * Np + n];
        S[0][1] = S[1][0] = sigma[2 * Np + n];
    } else {
        S[0][0] = sigma[0 * Np + n]; S[1][1] = sigma[1 * Np + n]; S[2][2] = sigma[2 * Np + n];
        S[0][1] = S[1][0] = sigma[3 * Np + n];
        S[0][2] = S[2][0] = sigma[4 * Np + n];
        S[1][2] = S[2][1] = sigma[5 * Np + n];
    }
    for (int c = 0; c < D; ++c) tr += S[c][c];
    Dual ddr(0.0);
    if (p.trace_full) ddr = -(tr - tr_prev[n]) * Dual(3.0 / D);
    const Dual drho = drho_raw + 0.5 * ddr;
    const Dual rho = Dual(p.rho0) + drho;
    Dual u[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
    for (int c = 0; c < D; ++c) u[c] = (j[c] + 0.5 * p.f[c]) / rho;
    for (int c = 0; c < D; ++c) S[c][c] -= tr / Dual((double)D);
    Dual uu(0.0);
    for (int c = 0; c < D; ++c) uu += u[c] * u[c];
    const double omega = 1.0 / p.tau_lb;
    const double fpre = 1.0 - 0.5 * omega;
    Dual Xf[3][3];
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) Xf[r][c] = -ddr * u[r] * u[c] + u[c] * p.f[r] + u[r] * p.f[c];
    Dual trX(0.0);
    for (int c = 0; c < D; ++c) trX += Xf[c][c];
    int x, y, z;
    node_xyz(ch, n, x, y, z);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cq[3] = {L::cx(q), L::cy(q), L::cz(q)};
        Dual cu(0.0), cf(0.0), cSc(0.0), cXc(0.0);
        for (int r = 0; r < D; ++r) {
            if (cq[r]) {
                cu += cq[r] * u[r];
                cf += cq[r] * p.f[r];
            }
            for (int c = 0; c < D; ++c)
                if (cq[r] && cq[c]) {
                    cSc += (cq[r] * cq[c]) * S[r][c];
                    cXc += (cq[r] * cq[c]) * Xf[r][c];
                }
        }
        const double wq = L::w(q);
        const Dual dneq = wq * (drho + rho * (3.0 * cu + 4.5 * (cu * cu - cs2 * uu)));
        const Dual Fq = wq * (-4.5 * omega * cSc + fpre * (ddr + 3.0 * cf + 4.5 * (cXc - cs2 * trX)));
        const Dual post = dn[q] - omega * (dn[q] - dneq) + Fq;
        int xd = x + cq[0];
        xd = xd < 0 ? ch.nx - 1 : (xd >= ch.nx ? 0 : xd);
        const int yd = y + cq[1];
        bool wall = yd < 0 || yd >= ch.ny;
        int zd = z + cq[2];
        if (D == 3) {
            if (ch.wall_z) wall = wall || zd < 0 || zd >= ch.nz;
            else zd = zd < 0 ? ch.nz - 1 : (zd >= ch.nz ? 0 : zd);
        }
        if (wall) dn_out[L::opp(q) * Np + n] = post;
        else dn_out[q * Np + (xd + ch.nx * (yd + ch.ny * zd))] = post;
    }
    rho_f[n] = drho;
    for (int c = 0; c < D; ++c) u_f[c * Np + n] = u[c];
    tr_prev[n] = p.trace_full ? tr : Dual(0.0);
}

// Value (k < 0) or derivative k of a dual field, gathered as doubles [comp][N] (+ offset on values).
__global__ void k_gather_t(const Dual* __restrict__ src, long long Npad, int ncomp, int N, int k, double offset,
                           double* __restrict__ dst) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)ncomp * N) return;
    const int c = (int)(i / N), n = (int)(i % N);
    const Dual& v = src[c * Npad + n];
    dst[i] = k < 0 ? v.v + offset : v.d[k];
}

// N1 = sigma_xx - sigma_yy, value or derivative k.
__global__ void k_n1_t(const Dual* __restrict__ sigma, long long Npad, int N, int k, double* __restrict__ dst) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const Dual a = sigma[n], b = sigma[Npad + n];
    dst[n] = k < 0 ? a.v - b.v : a.d[k] - b.d[k];
}

}  // namespace lbk
