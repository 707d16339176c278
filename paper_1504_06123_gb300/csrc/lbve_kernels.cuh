// lbve_kernels.cuh -- sm_103a kernels of one hybrid LB step (Sec. III of arXiv:1504.06123): the shared
// types, the moments, the finite-difference gradient and the stress history (sweep and commit, in FP32,
// FP64 and the 16-bit block-scaled form).  The collision kernel and the history-free instantaneous
// model are in lbve_collide.cuh.
//
// Per step, three launches on one stream:
//   k_moments        : u_raw = (sum c n + f/2) / sum n                                (Eq. hydrofields)
//   k_sweep          : every retained history point advances E <- exp(kappa(t-1)) E, forms
//                      -d_t'B = E kappa E^T + (.)^T and the modulus of Eq. (nlmax); partial trapezoidal
//                      sums of Eq. (gitt) per slot chunk.  This is the O(nodes x points) part and the
//                      only one that matters for bandwidth.
//   k_collide_stream : per node: kappa(t) by finite differences, sigma_struc(t) from the partials and the
//                      point created now, the block merges of the quasi-logarithmic grid and the new
//                      point; then trace split, density source, BGK collision with the forcing of
//                      Eq. (bodyforce), push streaming with half-way bounce-back.
//
// Layouts (device, structure of arrays, every plane padded to Npad nodes):
//   populations  d_n[q][Npad]   type P   stored as n_q - w_q rho0 (deviation form keeps FP32 exact
//                                        enough for velocities of 1e-5)
//   history      X[slot][c][Npad] type R X = E - 1 of each retained point (c < d*d, row-major)
//                K[slot][c][Npad] type R kappa of each retained point
//                part[chunk][i][Npad] type R partial sums of the sweep (scratch, rewritten every step)
//   node fields  (double; O(N) words, negligible traffic next to the history)
//                u_raw[d][Npad], kappa[d*d][Npad], sigma[nsig][Npad], tr_prev[Npad], drho[Npad] (rho - rho0),
//                u[d][Npad]
// P (population storage) and R (history storage and arithmetic) are float or double independently.
// slot = bb*C + ring index, bb = 0 (coarsest block) .. B-1 (finest).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "lbve_sched.cuh"

namespace lbk {

// ------------------------------------------------------------------------------------------------
// Velocity sets (Sec. III for D2Q9; standard D3Q19 for the duct).  cs^2 = 1/3.
// ------------------------------------------------------------------------------------------------
template <int Q> struct Lattice;

template <> struct Lattice<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int q) { return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int q) { return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int q) { return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
    __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 5 + 2) % 4) + 5); }
};

// D3Q19: 0 rest; 1..6 faces +x,-x,+y,-y,+z,-z; 7..18 edges.
template <> struct Lattice<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int c(int q, int a) {
        // faces
        return q == 0 ? 0
             : q <= 6 ? (((q - 1) / 2) == a ? (((q - 1) & 1) ? -1 : 1) : 0)
             : edge(q - 7, a);
    }
    // edges: for axis pairs (x,y), (x,z), (y,z), signs (+,+), (+,-), (-,+), (-,-)
    __host__ __device__ static constexpr int edge(int e, int a) {
        return (pair_a(e / 4) == a) ? ((e & 2) ? -1 : 1) : ((pair_b(e / 4) == a) ? ((e & 1) ? -1 : 1) : 0);
    }
    __host__ __device__ static constexpr int pair_a(int p) { return p == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int pair_b(int p) { return p == 0 ? 1 : 2; }
    __host__ __device__ static constexpr int cx(int q) { return c(q, 0); }
    __host__ __device__ static constexpr int cy(int q) { return c(q, 1); }
    __host__ __device__ static constexpr int cz(int q) { return c(q, 2); }
    __host__ __device__ static constexpr double w(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
    __host__ __device__ static constexpr int opp(int q) {
        return q == 0 ? 0 : (q <= 6 ? (((q - 1) ^ 1) + 1) : (((q - 7) ^ 3) + 7));
    }
};

// ------------------------------------------------------------------------------------------------
// Geometry and parameters shared by the kernels
// ------------------------------------------------------------------------------------------------
// One channel of a batch (a single channel is a batch of one).  Channels are stored one after the
// other: channel c owns nodes off .. off + nx*ny*nz - 1, x fastest.  Kept in device memory, so that
// changing a force or a parameter does not change any kernel argument (captured graphs stay valid).
struct Chan {
    int off;          // first node of the channel
    int nx, ny, nz;   // nodes per axis
    int wall_z;       // walls at z = -1/2, nz - 1/2
    int trace_full;   // Eq. (bodyforce) with the density source
    double rho0, tau_lb;
    double omega;     // BGK rate 1 / tau_lb
    double f[3];      // force density rho0 g
    double G_inf, inv_tau, inv_gc;
    int xbc;          // 1: pressure-step boundary along x
    double drho_gh;   // its ghost densities rho0 +- drho_gh (the linear profile of the pressure drop)
    // the same values rounded to float, for the node arithmetic of float populations
    float rho0_f, omega_f, f_f[3], G_inf_f, drho_gh_f;
};

// Node arithmetic type of the per-node kernels: the channel parameters in that type.
template <typename T> __device__ __forceinline__ T chan_val(double d, float f);
template <> __device__ __forceinline__ double chan_val<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float chan_val<float>(double, float f) { return f; }

// Tag of the node arithmetic a history commit sums and returns sigma_struc in (double with double
// populations, float with float populations).
template <typename N> struct Arith {};

struct Geom {
    int N;                 // all nodes of all channels
    long long Npad;        // plane stride (multiple of 128)
    int nchan;
    const Chan* ch;        // [nchan]
    const int* chan_of;    // [Npad] channel of every node (nullptr for a single channel)
};

__device__ __forceinline__ int chan_index(const Geom& g, long long n) { return g.chan_of ? g.chan_of[n] : 0; }

// Coordinates of node n inside its channel.
__device__ __forceinline__ void node_xyz(const Chan& c, int n, int& x, int& y, int& z) {
    const int l = n - c.off;
    x = l % c.nx;
    const int r = l / c.nx;
    y = r % c.ny;
    z = r / c.ny;
}

// ------------------------------------------------------------------------------------------------
// K1: raw moments -> u_raw
// ------------------------------------------------------------------------------------------------
// Zeroth and first moments of the (deviation-form) populations of one node in the type T.  In double the
// sums run in q order.  In float the terms can be far larger than the sums (the even, stress-carrying parts
// of opposite populations cancel in j, and their isotropic parts largely cancel in the mass), so the float
// sums are formed without cancellation error: j from differences of opposite populations (exact when the two
// are within a factor of two, i.e. when the even part dominates), the mass by compensated summation (each
// addition's rounding error recovered exactly by the two-sum identity and carried along).
template <int Q, typename T>
__device__ __forceinline__ void node_moments(const T* v, T& drho, T* j) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    drho = T(0);
    j[0] = j[1] = j[2] = T(0);
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            drho += v[q];
            if (L::cx(q)) j[0] += L::cx(q) * v[q];
            if (L::cy(q)) j[1] += L::cy(q) * v[q];
            if (D == 3 && L::cz(q)) j[2] += L::cz(q) * v[q];
        }
    } else {
        T c = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const T t = drho + v[q];
            const T z = t - drho;
            c += (drho - (t - z)) + (v[q] - z);
            drho = t;
        }
        drho += c;
#pragma unroll
        for (int q = 0; q < Q; ++q) {   // each pair (q, opposite of q) once, from its member with c_a = +1
            const T d = v[q] - v[L::opp(q)];
            if (L::cx(q) > 0) j[0] += d;
            if (L::cy(q) > 0) j[1] += d;
            if (D == 3 && L::cz(q) > 0) j[2] += d;
        }
    }
}

// The first kernel of a step also advances the device step counter (it starts at -1), so that the later
// kernels of the step all read the same t.
// M: arithmetic of the moments (float only for float populations with the 16-bit history); u_raw is stored
// in M as well (float values in the same buffer), which the collision's gradient then reads in M.
template <int Q, typename P, typename M>
__global__ void __launch_bounds__(256) k_moments(const P* __restrict__ dn, double* __restrict__ u_raw, Geom g,
                                                 long long* t_dev) {
    using L = Lattice<Q>;
    constexpr int D = L::D;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n == 0) *t_dev += 1;
    if (n >= g.N) return;
    const Chan& p = g.ch[chan_index(g, n)];
    M v[Q], drho, j[3];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = (M)dn[(long long)q * g.Npad + n];
    node_moments<Q, M>(v, drho, j);
    const M inv = M(1) / (chan_val<M>(p.rho0, p.rho0_f) + drho);
    M* const ur = reinterpret_cast<M*>(u_raw);
#pragma unroll
    for (int a = 0; a < D; ++a) ur[(long long)a * g.Npad + n] = (j[a] + M(0.5) * chan_val<M>(p.f[a], p.f_f[a])) * inv;
}

// ------------------------------------------------------------------------------------------------
// kappa(t) by second-order finite differences of u_raw (Sec. III): central in the bulk and on
// periodic axes; at a wall-adjacent node the derivative of the parabola through the no-slip wall
// half a node away and the two nearest nodes: low wall u0 + u1/3, high wall -(u0 + u_{-1}/3).
// ------------------------------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ real d_axis(real um, real u0, real up, int i, int n, bool periodic) {
    if (periodic) return real(0.5) * (up - um);
    if (i == 0) return u0 + up * real(1.0 / 3.0);
    if (i == n - 1) return -(u0 + um * real(1.0 / 3.0));
    return real(0.5) * (up - um);
}

template <int D, typename real>
__device__ __forceinline__ void kappa_fd(const real* __restrict__ u, long long Npad, const Chan& c, int n, real* kap) {
    int x, y, z;
    node_xyz(c, n, x, y, z);
    const int xm = (x == 0 ? c.nx - 1 : x - 1), xp = (x == c.nx - 1 ? 0 : x + 1);
    const int ym = (y == 0 ? y : y - 1), yp = (y == c.ny - 1 ? y : y + 1);
    const int nxm = c.off + xm + c.nx * (y + c.ny * z), nxp = c.off + xp + c.nx * (y + c.ny * z);
    const int nym = c.off + x + c.nx * (ym + c.ny * z), nyp = c.off + x + c.nx * (yp + c.ny * z);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const real* ua = u + (long long)a * Npad;
        const real u0 = ua[n];
        kap[a * D + 0] = d_axis(ua[nxm], u0, ua[nxp], x, c.nx, true);
        kap[a * D + 1] = d_axis(ua[nym], u0, ua[nyp], y, c.ny, false);
    }
    if (D == 3) {
        int zm, zp;
        if (c.wall_z) { zm = (z == 0 ? z : z - 1); zp = (z == c.nz - 1 ? z : z + 1); }
        else { zm = (z == 0 ? c.nz - 1 : z - 1); zp = (z == c.nz - 1 ? 0 : z + 1); }
        const int nzm = c.off + x + c.nx * (y + c.ny * zm), nzp = c.off + x + c.nx * (y + c.ny * zp);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const real* ua = u + (long long)a * Npad;
            kap[a * D + (D - 1)] = d_axis(ua[nzm], ua[n], ua[nzp], z, c.nz, !c.wall_z);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Small matrix algebra in registers
// ------------------------------------------------------------------------------------------------
// A = exp(K) - 1 by the Taylor series in Horner form, truncated after K^4/4! (float: |K| <= 1e-2
// leaves < 1e-12) or K^8/8! (double).
template <int D, typename real>
__device__ __forceinline__ void expm1_mat(const real* K, real* A) {
    constexpr int DD = D * D;
    constexpr int ORDER = sizeof(real) == 4 ? 4 : 8;
    real P[DD];
#pragma unroll
    for (int i = 0; i < DD; ++i) P[i] = K[i] * real(1.0 / ORDER);   // K/ORDER
#pragma unroll
    for (int m = ORDER - 1; m >= 1; --m) {
        // P <- K (1 + P) / m
        real T[DD];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                real s = K[r * D + c];
#pragma unroll
                for (int k = 0; k < D; ++k) s += K[r * D + k] * P[k * D + c];
                T[r * D + c] = s * real(1.0 / m);
            }
#pragma unroll
        for (int i = 0; i < DD; ++i) P[i] = T[i];
    }
#pragma unroll
    for (int i = 0; i < DD; ++i) A[i] = P[i];
}

// The integrand of one history point with E = 1 + X: w G(age) (E kappa E^T + (E kappa E^T)^T), G of
// Eq. (nlmax) without the factor G_inf, accumulated into acc (nsig packed components).
template <typename real> struct FastMath {
    // exp(-x) and sqrt(x) as used by the integrand (double: the library functions)
    __device__ static __forceinline__ real exp_neg(real x) { return exp(-x); }
    __device__ static __forceinline__ real sqrt_pos(real x) { return sqrt(x); }
};
template <> struct FastMath<float> {
    // single-precision hardware approximations (2 ulp): exp(-x) = 2^(-x log2 e); sqrt(x) = x rsqrt(x)
    __device__ static __forceinline__ float exp_neg(float x) { return exp2f(-1.4426950408889634f * x); }
    __device__ static __forceinline__ float sqrt_pos(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
};

// The integrand of Eq. (gitt) at one point, added to acc (symmetric components xx, yy, [zz,] xy, [xz, yz]):
// w G(t, t') (E kap E^T + (E kap E^T)^T) = w G E Dm E^T with the rate of strain Dm = kap + kap^T, formed as
// F = E Dm = Dm + X Dm, then the upper triangle of F E^T = F + F X^T.
// WM = true: the White-Metzner form (Sec. II): the second exponential of Eq. (nlmax) takes the strain
// accumulated since the point was created, `strain`, instead of age * gammadot(point).
template <int D, typename real, bool WM = false>
__device__ __forceinline__ void point_integrand(const real* X, const real* kap, real age, real w,
                                                real inv_tau, real inv_gc, real* acc, real strain = real(0)) {
    constexpr int DD = D * D;
    real Dm[DD];
#pragma unroll
    for (int r = 0; r < D; ++r) {
        Dm[r * D + r] = kap[r * D + r] + kap[r * D + r];
#pragma unroll
        for (int c = r + 1; c < D; ++c) Dm[r * D + c] = Dm[c * D + r] = kap[r * D + c] + kap[c * D + r];
    }
    real F[DD];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            real s = Dm[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s += X[r * D + k] * Dm[k * D + c];
            F[r * D + c] = s;
        }
    auto S = [&](int r, int c) {   // (F E^T)_rc
        real s = F[r * D + c];
#pragma unroll
        for (int k = 0; k < D; ++k) s += F[r * D + k] * X[c * D + k];
        return s;
    };
    real gw;
    if (WM) {
        gw = w * FastMath<real>::exp_neg(age * inv_tau + strain * inv_gc);
    } else {
        // local shear rate of the point: gammadot^2 = (1/2) tr Dm^2
        real h = 0;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            h += real(0.5) * Dm[r * D + r] * Dm[r * D + r];
#pragma unroll
            for (int c = r + 1; c < D; ++c) h += Dm[r * D + c] * Dm[r * D + c];
        }
        const real gd = FastMath<real>::sqrt_pos(h);
        gw = w * FastMath<real>::exp_neg(age * (inv_tau + gd * inv_gc));
    }
    if (D == 2) {
        acc[0] += gw * S(0, 0);
        acc[1] += gw * S(1, 1);
        acc[2] += gw * S(0, 1);
    } else {
        acc[0] += gw * S(0, 0);
        acc[1] += gw * S(1, 1);
        acc[2] += gw * S(2, 2);
        acc[3] += gw * S(0, 1);
        acc[4] += gw * S(0, 2);
        acc[5] += gw * S(1, 2);
    }
}

// One history point of the in-place storage: advance X <- X + A + A X (E <- exp(kappa(t-1)) E), then
// its integrand.
template <int D, typename real, bool WM = false>
__device__ __forceinline__ void point_update(real* X, const real* A, const real* kap, real age, real w,
                                             real inv_tau, real inv_gc, real* acc, real strain = real(0)) {
    constexpr int DD = D * D;
    real Xn[DD];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            real s = X[r * D + c] + A[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s += A[r * D + k] * X[k * D + c];
            Xn[r * D + c] = s;
        }
#pragma unroll
    for (int i = 0; i < DD; ++i) X[i] = Xn[i];
    point_integrand<D, real, WM>(X, kap, age, w, inv_tau, inv_gc, acc, strain);
}

// ------------------------------------------------------------------------------------------------
// K2: the stress history sweep
// ------------------------------------------------------------------------------------------------
// VN consecutive values of one component plane, loaded and stored as one vector (16 bytes for
// 4 floats or 2 doubles).
template <typename R, int VN> struct alignas(sizeof(R) * VN) Vec { R v[VN]; };

template <typename R> struct SweepArgs {
    R* __restrict__ X;                // [L][DD][Npad]  E - 1
    const R* __restrict__ K;          // [L][DD][Npad]  kappa of each point (read only in the sweep)
    R* __restrict__ part;             // [S][NS][Npad]  partial trapezoid sums per slot chunk (scratch)
    const long long* t_dev;           // step index t
    int B, C, S;                      // grid shape; S slot chunks
    int cta_tasks;                    // 0: a task is one warp's; 1: a task is one CTA's (warps split its chunk)
    // White-Metzner form only: accumulated strain Gamma(t) = sum_{s<t} gammadot(s) of every node and the
    // value Gamma(t') each point was created with; a point's strain is their difference
    const double* __restrict__ gam_node;   // [Npad]
    const double* __restrict__ gam_pt;     // [L][Npad]
};

// Shared memory of the sweeps: per slot age, weight, partner (L entries each) + the per-block state; k_sweep
// adds (CTA tasks) the per-warp partial sums of one tile: 8 warps x NS x 32 VN values = 12 KB in every
// lattice / precision combination (NS VN sizeof(R) = 48).
__host__ __device__ inline size_t sweep_smem_bytes(int L) {
    return ((size_t)L * 12 + sizeof(BlockStep) * LBVE_MAXB + 15) / 16 * 16;
}
constexpr size_t kSweepRedBytes = 8 * 32 * 48;
__host__ __device__ inline size_t sweep_cta_smem_bytes(int L) { return sweep_smem_bytes(L) + kSweepRedBytes; }

// Slots [l0, l1) of the nodes n0 .. n0+VN-1 of one lane: advance every point in place,
// X <- X + A + A X with A = exp(kappa(t-1)) - 1 (Eq. eeval, newest factor on the left), and add
// w G (E kappa E^T + (.)^T) to acc.  The older half of a merge uses the average of the two kappa
// (Sec. III); the newer half (weight 0) is skipped.
template <int D, typename R, int VN, bool WM>
__device__ __forceinline__ void sweep_range(const SweepArgs<R>& a, const Geom& g, const float* s_age,
                                            const float* s_w, const int* s_part, long long s_last, long long n0,
                                            int l0, int l1, R (&acc)[VN][D == 2 ? 3 : 6]) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    using V = Vec<R, VN>;
    const long long Np = g.Npad;
    // relaxation rates of each node's channel (Eq. nlmax)
    R inv_tau[VN], inv_gc[VN];
#pragma unroll
    for (int j = 0; j < VN; ++j) {
        const Chan& c = g.ch[chan_index(g, n0 + j)];
        inv_tau[j] = (R)c.inv_tau;
        inv_gc[j] = (R)c.inv_gc;
    }
    // A = exp(kappa(t-1)) - 1 per node; kappa(t-1) is the point created last step (newest slot of the
    // finest block; a rest point before the first step)
    R A[VN][DD];
    {
        R kp[VN][DD];
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            const V v = *reinterpret_cast<const V*>(a.K + (s_last * DD + c) * Np + n0);
#pragma unroll
            for (int j = 0; j < VN; ++j) kp[j][c] = v.v[j];
        }
#pragma unroll
        for (int j = 0; j < VN; ++j) expm1_mat<D>(kp[j], A[j]);
    }
#pragma unroll
    for (int j = 0; j < VN; ++j)
#pragma unroll
        for (int i = 0; i < NS; ++i) acc[j][i] = 0;
    using VD = Vec<double, VN>;
    VD gam_now;
    if (WM) gam_now = *reinterpret_cast<const VD*>(a.gam_node + n0);

    for (int l = l0; l < l1; ++l) {
        const float w = s_w[l];
        if (w == 0.0f) continue;                 // same slot for the whole warp: uniform branch
        R* Xp = a.X + (long long)l * DD * Np + n0;
        const R* Kp = a.K + (long long)l * DD * Np + n0;
        R X[VN][DD], kap[VN][DD];
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            const V xv = *reinterpret_cast<const V*>(Xp + c * Np);
            const V kv = *reinterpret_cast<const V*>(Kp + c * Np);
#pragma unroll
            for (int j = 0; j < VN; ++j) { X[j][c] = xv.v[j]; kap[j][c] = kv.v[j]; }
        }
        const int part = s_part[l];
        if (part >= 0) {   // older half of a merge: kappa averaged with the newer half
            const R* K2 = a.K + (long long)part * DD * Np + n0;
#pragma unroll
            for (int c = 0; c < DD; ++c) {
                const V kv = *reinterpret_cast<const V*>(K2 + c * Np);
#pragma unroll
                for (int j = 0; j < VN; ++j) kap[j][c] = R(0.5) * (kap[j][c] + kv.v[j]);
            }
        }
        const R age = (R)s_age[l], wr = (R)w;
        R strain[VN];
        if (WM) {   // a merged point keeps the older half's creation strain (its slot l)
            const VD gp = *reinterpret_cast<const VD*>(a.gam_pt + (long long)l * Np + n0);
#pragma unroll
            for (int j = 0; j < VN; ++j) strain[j] = (R)(gam_now.v[j] - gp.v[j]);
        }
#pragma unroll
        for (int j = 0; j < VN; ++j)
            point_update<D, R, WM>(X[j], A[j], kap[j], age, wr, inv_tau[j], inv_gc[j], acc[j], WM ? strain[j] : R(0));
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            V xv;
#pragma unroll
            for (int j = 0; j < VN; ++j) xv.v[j] = X[j][c];
            *reinterpret_cast<V*>(Xp + c * Np) = xv;
        }
    }
}

// Persistent sweep over tasks (tile of 32*VN consecutive nodes, chunk of consecutive slots).  Lane i
// handles nodes tile*32*VN + i*VN ... + VN-1, so every component plane is read and written with one
// 16-byte access per lane and 512 contiguous bytes per warp.
//  - warp tasks (cta_tasks = 0): each warp takes whole tasks and writes its chunk's partial sum;
//  - CTA tasks (cta_tasks = 1): the CTA's warps take consecutive pieces of one task's chunk, and their
//    sums are added in warp order through shared memory: a chunk count S then keeps 8x the warps busy
//    that warp tasks would (few nodes: full occupancy without S-fold partial sums in the commit).
// Each task writes its partial sum of w G (E kappa E^T + (.)^T) to `part`; k_collide_stream (or
// k_commit) adds the chunks in a fixed order, so the result does not depend on scheduling.
template <int D, typename R, int VN, bool WM = false>
__global__ void __launch_bounds__(256, 2) k_sweep(SweepArgs<R> a, Geom g) {
    constexpr int NS = D == 2 ? 3 : 6;
    using V = Vec<R, VN>;
    const int L = a.B * a.C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_age = reinterpret_cast<float*>(smem_raw);
    float* s_w = s_age + L;
    int* s_part = reinterpret_cast<int*>(s_w + L);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(s_part + L);
    R* s_red = reinterpret_cast<R*>(smem_raw + sweep_smem_bytes(L));

    const long long t = *a.t_dev;
    sched_step_cta(a.B, a.C, t, s_bs);
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int age, part;
        const float w = sched_slot_role(s_bs, a.C, l / a.C, l % a.C, &age, &part);
        s_age[l] = (float)age;
        s_w[l] = w;
        s_part[l] = part;
    }
    __syncthreads();

    const long long Np = g.Npad;
    const int lane = threadIdx.x & 31;
    const int tiles = (int)(Np / (32 * VN));
    const int tasks = tiles * a.S;
    const int chunk_len = (L + a.S - 1) / a.S;
    const long long s_last = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_prev;
    R acc[VN][NS];

    if (!a.cta_tasks) {
        const int gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        const int nwarps = gridDim.x * (blockDim.x >> 5);
        for (int task = gwarp; task < tasks; task += nwarps) {
            const int tile = task % tiles;
            const int chunk = task / tiles;
            const long long n0 = (long long)tile * 32 * VN + lane * VN;
            const int l0 = chunk * chunk_len;
            sweep_range<D, R, VN, WM>(a, g, s_age, s_w, s_part, s_last, n0, l0, min(L, l0 + chunk_len), acc);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                V v;
#pragma unroll
                for (int j = 0; j < VN; ++j) v.v[j] = acc[j][i];
                *reinterpret_cast<V*>(a.part + ((long long)chunk * NS + i) * Np + n0) = v;
            }
        }
        return;
    }
    const int nw = blockDim.x >> 5;                 // warps of the CTA (8: the shared buffer's size)
    const int wib = threadIdx.x >> 5;
    const int sub_len = (chunk_len + nw - 1) / nw;
    constexpr int TN = 32 * VN;                     // nodes of a tile
    for (int task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int tile = task % tiles;
        const int chunk = task / tiles;
        const long long n0 = (long long)tile * TN + lane * VN;
        const int c0 = chunk * chunk_len, c1 = min(L, c0 + chunk_len);
        const int l0 = min(c1, c0 + wib * sub_len);
        sweep_range<D, R, VN, WM>(a, g, s_age, s_w, s_part, s_last, n0, l0, min(c1, l0 + sub_len), acc);
#pragma unroll
        for (int i = 0; i < NS; ++i)
#pragma unroll
            for (int j = 0; j < VN; ++j) s_red[(wib * NS + i) * TN + lane * VN + j] = acc[j][i];
        __syncthreads();
        for (int k = threadIdx.x; k < NS * TN; k += blockDim.x) {
            const int i = k / TN, m = k - i * TN;
            R sum = s_red[i * TN + m];
            for (int w = 1; w < nw; ++w) sum += s_red[(w * NS + i) * TN + m];
            a.part[((long long)chunk * NS + i) * Np + (long long)tile * TN + m] = sum;
        }
        __syncthreads();
    }
}

// Autotuning aid: the commit's read of the chunk partials (one thread per node, chunks in order), so
// that the tuner weighs a slot-chunk count S by the sweep plus the reduction it causes in the commit (A: the
// commit's summation type).
template <typename R, typename A>
__global__ void k_part_read(const R* __restrict__ part, int S, int NS, long long Np, int N, double* sink) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    A acc = A(0);
#pragma unroll 4
    for (int c = 0; c < S; ++c)
        for (int i = 0; i < NS; ++i) acc += (A)part[((long long)c * NS + i) * Np + n];
    if (acc == A(1.2345e30)) *sink = (double)acc;   // keeps the loads; the all-rest history sums to 0
}

// ------------------------------------------------------------------------------------------------
// History commit of one node (after the sweep): sigma_struc(t) from the chunk partials plus the point
// created now (age 0, E = 1, weight 1/2, modulus G_inf), then the block merges (coarsest first, so every
// ring slot is read before it is overwritten) and the new point entering the finest block.
// ------------------------------------------------------------------------------------------------
template <typename R> struct CommitArgs {
    R* __restrict__ X;
    R* __restrict__ K;
    const R* __restrict__ part;       // [S][NS][Npad]
    int B, C, S;
    double* __restrict__ gam_node;    // White-Metzner form: Gamma(t) per node [Npad] (nullptr: nlM)
    double* __restrict__ gam_pt;      //                     Gamma(t') per point [L][Npad]
};

// Local shear rate of Sec. II, gammadot = sqrt((1/2) tr D^2), D = kappa + kappa^T (double).
template <int D>
__device__ __forceinline__ double shear_rate_d(const double* k) {
    double trD2 = 0;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const double v = k[r * D + c] + k[c * D + r];
            trD2 += v * v;
        }
    return sqrt(0.5 * trD2);
}

template <int D, typename R, typename N>
__device__ __forceinline__ void hist_commit(const CommitArgs<R>& a, const BlockStep* s_bs, long long Np, int n,
                                            const double* ktd, N G_inf, N* sig /* [NS] out */) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    N acc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i] = N(0);
#pragma unroll 4
    for (int c = 0; c < a.S; ++c)
#pragma unroll
        for (int i = 0; i < NS; ++i) acc[i] += (N)a.part[((long long)c * NS + i) * Np + n];
    // the new point, summed in the history's precision like every other point
    R kt[DD];
#pragma unroll
    for (int c = 0; c < DD; ++c) kt[c] = (R)ktd[c];
    if (D == 2) {
        acc[0] += (N)(R(0.5) * (kt[0] + kt[0]));
        acc[1] += (N)(R(0.5) * (kt[3] + kt[3]));
        acc[2] += (N)(R(0.5) * (kt[1] + kt[2]));
    } else {
        acc[0] += (N)(R(0.5) * (kt[0] + kt[0]));
        acc[1] += (N)(R(0.5) * (kt[4] + kt[4]));
        acc[2] += (N)(R(0.5) * (kt[8] + kt[8]));
        acc[3] += (N)(R(0.5) * (kt[1] + kt[3]));
        acc[4] += (N)(R(0.5) * (kt[2] + kt[6]));
        acc[5] += (N)(R(0.5) * (kt[5] + kt[7]));
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) sig[i] = G_inf * acc[i];

    for (int bb = 1; bb < a.B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long src1 = (long long)bb * a.C + o1, src2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            a.X[(dst * DD + c) * Np + n] = a.X[(src1 * DD + c) * Np + n];
            a.K[(dst * DD + c) * Np + n] = R(0.5) * (a.K[(src1 * DD + c) * Np + n] + a.K[(src2 * DD + c) * Np + n]);
        }
        if (a.gam_pt) a.gam_pt[dst * Np + n] = a.gam_pt[src1 * Np + n];   // older time, older strain origin
    }
    const long long dst = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
#pragma unroll
    for (int c = 0; c < DD; ++c) {
        a.X[(dst * DD + c) * Np + n] = R(0);
        a.K[(dst * DD + c) * Np + n] = kt[c];
    }
    if (a.gam_pt) {   // the new point starts at Gamma(t); the node moves on by the strain of [t, t+1]
        const double gnow = a.gam_node[n];
        a.gam_pt[dst * Np + n] = gnow;
        a.gam_node[n] = gnow + shear_rate_d<D>(ktd);
    }
}

// Uniform entry for every history storage: kprev = kappa(t-1) of the node (the node kappa field before
// this step overwrites it), used by storages that keep a per-node frame; sigma_struc(t) summed and returned
// in the node arithmetic N.
template <int D, typename R, typename N>
__device__ __forceinline__ void hist_commit_any(Arith<N>, const CommitArgs<R>& a, const BlockStep* s_bs, long long Np,
                                                int n, const double* /*kprev*/, const double* ktd, const Chan& p,
                                                N* sig, long long /*t*/) {
    hist_commit<D, R, N>(a, s_bs, Np, n, ktd, chan_val<N>(p.G_inf, p.G_inf_f), sig);
}

// ------------------------------------------------------------------------------------------------
// Reduced-precision history (precision variant): 16-bit block-scaled storage in a per-node frame.
//
// Every node keeps a frame R(t) = E(t, t_b), the deformation since the last rebase step t_b, in FP32
// (Rm = R - 1).  Every point keeps Q = E(t_b, t') (or R(t')^-1 for points created after t_b), so that
// E(t, t') = R(t) Q: the per-step left multiplication by exp(kappa(t-1)) of Eq. (eeval) acts on the
// node's frame only, and the points are read, not rewritten.  Every TB steps the sweep rewrites each
// point's Q as E(t, t') and the frame restarts at 1, which bounds the strain carried by the frame.
// Q - 1 and kappa are stored as block-scaled 16-bit vectors: d*d int16 mantissas m_c sharing one
// power-of-two exponent e, value_c = m_c 2^e, |m_c| <= 32767 (relative precision 2^-15 of the largest
// component).  Values are written once (kappa; Q between rebases) and re-rounded only at rebases.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }   // -126 <= k <= 127

// Stored form of a block-scaled vector: unsigned halves u_c = m_c + 32768 and the exponent byte
// eb = e + 127 (eb = 0 for the zero vector), so that all-zero bytes decode to 0 (a rest point) and the
// scale 2^e is the float whose exponent field is eb.
template <int DD>
__device__ __forceinline__ void s16_encode(const float* v, unsigned short* u, unsigned char* eb) {
    float mx = 0.0f;
#pragma unroll
    for (int c = 0; c < DD; ++c) mx = fmaxf(mx, fabsf(v[c]));
    if (!(mx > 0.0f)) {
#pragma unroll
        for (int c = 0; c < DD; ++c) u[c] = 32768;
        *eb = 0;
        return;
    }
    int ex = 0;
    frexpf(fminf(mx, 3.0e38f), &ex);                              // mx = f 2^ex, 0.5 <= f < 1
    const int es = min(126, max(-126, ex - 15));                 // |v| < 2^ex  =>  |v| 2^-es < 2^15
    const float inv = pow2f(-es);
#pragma unroll
    for (int c = 0; c < DD; ++c)
        u[c] = (unsigned short)(32768 + (int)fminf(32767.0f, fmaxf(-32767.0f, rintf(v[c] * inv))));
    *eb = (unsigned char)(es + 127);
}

__device__ __forceinline__ float s16_scale(unsigned eb) { return __int_as_float((int)(eb << 23)); }

template <int DD>
__device__ __forceinline__ void s16_decode(const unsigned short* u, unsigned eb, float* v) {
    const float sc = s16_scale(eb);
#pragma unroll
    for (int c = 0; c < DD; ++c) v[c] = (float)((int)u[c] - 32768) * sc;
}

// Decode of packed halves without int->float conversions: a half u placed under the exponent of
// 1.5 * 2^23 is the float 12582912 + u exactly; f sc - 12615680 sc = (u - 32768) sc is then exact (at
// most 16 significant bits) in one FMA.
struct S16Scale {
    float sc, c1;
    S16Scale() = default;
    __device__ __forceinline__ explicit S16Scale(unsigned eb) : sc(s16_scale(eb)), c1(-12615680.0f * s16_scale(eb)) {}
};
__device__ __forceinline__ float s16_lo(unsigned w, const S16Scale& s) {
    return fmaf(__int_as_float((int)__byte_perm(w, 0x4B40u, 0x5410)), s.sc, s.c1);
}
__device__ __forceinline__ float s16_hi(unsigned w, const S16Scale& s) {
    return fmaf(__int_as_float((int)__byte_perm(w, 0x4B40u, 0x5432)), s.sc, s.c1);
}
__device__ __forceinline__ unsigned s16_exp(unsigned word, int j) { return (word >> (8 * j)) & 0xFFu; }

struct CommitS16 {
    unsigned short* __restrict__ Qm; // [L][DD][Npad] biased mantissas of Q - 1
    unsigned char* __restrict__ Qe;  // [L][Npad] biased exponents
    unsigned short* __restrict__ Km; // [L][DD][Npad] biased mantissas of kappa
    unsigned char* __restrict__ Ke;  // [L][Npad]
    float* __restrict__ Rm;          // [DD][Npad] frame R - 1 of each node
    const float* __restrict__ part;  // [S][NS][Npad]
    int B, C, S, TB;
};

// History storages whose node sums may run in float with float populations (the 16-bit forms).
template <class H> struct Hist16 { static constexpr bool value = false; };
template <> struct Hist16<CommitS16> { static constexpr bool value = true; };

// R - 1 of the frame after step t: exp(kappa(t-1)) R(t-1) - 1 = A + Rm + A Rm.
template <int D>
__device__ __forceinline__ void frame_advance(const double* kprev, const float* Rm, float* Rn) {
    constexpr int DD = D * D;
    float kp[DD], A[DD];
#pragma unroll
    for (int c = 0; c < DD; ++c) kp[c] = (float)kprev[c];
    expm1_mat<D>(kp, A);
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float s = Rm[r * D + c] + A[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s += A[r * D + k] * Rm[k * D + c];
            Rn[r * D + c] = s;
        }
}

// Q - 1 of a point created now, Q = R^-1: with R = 1 + M, R^-1 - 1 = -R^-1 M (no cancellation).
template <int D>
__device__ __forceinline__ void frame_inverse_dev(const float* M, float* X) {
    float Ri[D * D];
    if (D == 2) {
        const float a = 1.0f + M[0], b = M[1], c = M[2], d = 1.0f + M[3];
        const float det = a * d - b * c;
        Ri[0] = d / det; Ri[1] = -b / det; Ri[2] = -c / det; Ri[3] = a / det;
    } else {
        float R[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) R[i] = M[i] + ((i % 4 == 0) ? 1.0f : 0.0f);
        const float c00 = R[4] * R[8] - R[5] * R[7], c01 = R[5] * R[6] - R[3] * R[8], c02 = R[3] * R[7] - R[4] * R[6];
        const float det = R[0] * c00 + R[1] * c01 + R[2] * c02;
        Ri[0] = c00 / det; Ri[3] = c01 / det; Ri[6] = c02 / det;
        Ri[1] = (R[2] * R[7] - R[1] * R[8]) / det; Ri[4] = (R[0] * R[8] - R[2] * R[6]) / det;
        Ri[7] = (R[1] * R[6] - R[0] * R[7]) / det;
        Ri[2] = (R[1] * R[5] - R[2] * R[4]) / det; Ri[5] = (R[2] * R[3] - R[0] * R[5]) / det;
        Ri[8] = (R[0] * R[4] - R[1] * R[3]) / det;
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float s = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) s -= Ri[r * D + k] * M[k * D + c];
            X[r * D + c] = s;
        }
}

// sigma of a node from the frame-free sum: the sweep accumulates P = sum w G (Q kappa Q^T + (.)^T) (packed
// symmetric, NS components); since every point of the node sees the same frame, the sum with
// E = R Q is R P R^T.
template <int D, typename N>
__device__ __forceinline__ void frame_apply(const float* Rm, const N* p, N* out) {
    N P[D][D], R[D][D], RP[D][D];
    if (D == 2) {
        P[0][0] = p[0]; P[1][1] = p[1]; P[0][1] = P[1][0] = p[2];
    } else {
        P[0][0] = p[0]; P[1][1] = p[1]; P[2][2] = p[2];
        P[0][1] = P[1][0] = p[3]; P[0][2] = P[2][0] = p[4]; P[1][2] = P[2][1] = p[5];
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) R[r][c] = (N)Rm[r * D + c] + (r == c ? N(1) : N(0));
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            N acc = N(0);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += R[r][k] * P[k][c];
            RP[r][c] = acc;
        }
    N S[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            N acc = N(0);
#pragma unroll
            for (int k = 0; k < D; ++k) acc += RP[r][k] * R[c][k];
            S[r][c] = acc;
        }
    if (D == 2) {
        out[0] = S[0][0]; out[1] = S[1][1]; out[2] = S[0][1];
    } else {
        out[0] = S[0][0]; out[1] = S[1][1]; out[2] = S[2][2];
        out[3] = S[0][1]; out[4] = S[0][2]; out[5] = S[1][2];
    }
}

template <int D, typename N, typename K>
__device__ __forceinline__ void hist_commit_any(Arith<N>, const CommitS16& a, const BlockStep* s_bs, long long Np,
                                                int n, const double* kprev, const K* ktd, const Chan& p,
                                                N* sig, long long t) {
    const N G_inf = chan_val<N>(p.G_inf, p.G_inf_f);
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    // the frame of this step (identical arithmetic to the sweep's rebase path), then the rebase
    float Rm[DD], Rn[DD];
#pragma unroll
    for (int c = 0; c < DD; ++c) Rm[c] = a.Rm[c * Np + n];
    frame_advance<D>(kprev, Rm, Rn);
    const bool rebase = (t % a.TB) == 0;
    // sigma: R (sum of chunk partials) R^T + the point created now (its stored, rounded kappa; E = 1,
    // weight 1/2)
    N acc[NS], P[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) P[i] = N(0);
#pragma unroll 4
    for (int c = 0; c < a.S; ++c)
#pragma unroll
        for (int i = 0; i < NS; ++i) P[i] += (N)a.part[((long long)c * NS + i) * Np + n];
    frame_apply<D, N>(Rn, P, acc);
    float kt[DD];
    unsigned short km[DD];
    unsigned char ke;
#pragma unroll
    for (int c = 0; c < DD; ++c) kt[c] = (float)ktd[c];
    s16_encode<DD>(kt, km, &ke);
    s16_decode<DD>(km, ke, kt);
    if (D == 2) {
        acc[0] += (N)(0.5f * (kt[0] + kt[0]));
        acc[1] += (N)(0.5f * (kt[3] + kt[3]));
        acc[2] += (N)(0.5f * (kt[1] + kt[2]));
    } else {
        acc[0] += (N)(0.5f * (kt[0] + kt[0]));
        acc[1] += (N)(0.5f * (kt[4] + kt[4]));
        acc[2] += (N)(0.5f * (kt[8] + kt[8]));
        acc[3] += (N)(0.5f * (kt[1] + kt[3]));
        acc[4] += (N)(0.5f * (kt[2] + kt[6]));
        acc[5] += (N)(0.5f * (kt[5] + kt[7]));
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) sig[i] = G_inf * acc[i];
#pragma unroll
    for (int c = 0; c < DD; ++c) {
        if (rebase) Rn[c] = 0.0f;
        a.Rm[c * Np + n] = Rn[c];
    }
    // block merges, coarsest first: the older point's Q moves, kappa is averaged and re-encoded
    for (int bb = 1; bb < a.B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long src1 = (long long)bb * a.C + o1, src2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
        unsigned short m1[DD], m2[DD], mo[DD];
        float k1[DD], k2[DD];
        unsigned char eo;
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            a.Qm[(dst * DD + c) * Np + n] = a.Qm[(src1 * DD + c) * Np + n];
            m1[c] = a.Km[(src1 * DD + c) * Np + n];
            m2[c] = a.Km[(src2 * DD + c) * Np + n];
        }
        a.Qe[dst * Np + n] = a.Qe[src1 * Np + n];
        s16_decode<DD>(m1, a.Ke[src1 * Np + n], k1);
        s16_decode<DD>(m2, a.Ke[src2 * Np + n], k2);
#pragma unroll
        for (int c = 0; c < DD; ++c) k1[c] = 0.5f * (k1[c] + k2[c]);
        s16_encode<DD>(k1, mo, &eo);
#pragma unroll
        for (int c = 0; c < DD; ++c) a.Km[(dst * DD + c) * Np + n] = mo[c];
        a.Ke[dst * Np + n] = eo;
    }
    // the new point: Q = R^-1 of the frame after this step, kappa(t)
    const long long dst = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
    float X[DD];
    unsigned short qm[DD];
    unsigned char qe;
    frame_inverse_dev<D>(Rn, X);
    s16_encode<DD>(X, qm, &qe);
#pragma unroll
    for (int c = 0; c < DD; ++c) {
        a.Qm[(dst * DD + c) * Np + n] = qm[c];
        a.Km[(dst * DD + c) * Np + n] = km[c];
    }
    a.Qe[dst * Np + n] = qe;
    a.Ke[dst * Np + n] = ke;
}

// Sweep of the 16-bit history: lanes hold VN consecutive nodes (one 32-bit word of exponents and VN/2
// words of mantissas per plane), tasks as in k_sweep.  Each point contributes with Q in place of E
// (the frame is applied once per node in the commit); on rebase steps the point's Q is rewritten as
// E(t, t') = R Q with the frame of this step.
template <int D, int VN>
__global__ void __launch_bounds__(256, 2) k_sweep_s16(CommitS16 a, const double* __restrict__ kprev,
                                                      const long long* t_dev, Geom g) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    static_assert(VN == 2 || VN == 4, "packed decode handles 2 or 4 nodes per lane");
    using VW = Vec<unsigned, VN / 2>;
    using VF = Vec<float, VN>;
    using VS = Vec<unsigned short, VN>;
    using VE = Vec<unsigned char, VN>;
    const int L = a.B * a.C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* s_age = reinterpret_cast<float*>(smem_raw);
    float* s_w = s_age + L;
    int* s_part = reinterpret_cast<int*>(s_w + L);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(s_part + L);

    const long long t = *t_dev;
    sched_step_cta(a.B, a.C, t, s_bs);
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int age, part;
        const float w = sched_slot_role(s_bs, a.C, l / a.C, l % a.C, &age, &part);
        s_age[l] = (float)age;
        s_w[l] = w;
        s_part[l] = part;
    }
    __syncthreads();

    const long long Np = g.Npad;
    const int lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int tiles = (int)(Np / (32 * VN));
    const int tasks = tiles * a.S;
    const int chunk_len = (L + a.S - 1) / a.S;
    const bool rebase = (t % a.TB) == 0;

    for (int task = gwarp; task < tasks; task += nwarps) {
        const int tile = task % tiles;
        const int chunk = task / tiles;
        const long long n0 = (long long)tile * 32 * VN + lane * VN;
        float inv_tau[VN], inv_gc[VN];
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            const Chan& c = g.ch[chan_index(g, n0 + j)];
            inv_tau[j] = (float)c.inv_tau;
            inv_gc[j] = (float)c.inv_gc;
        }
        float F[VN][DD];   // frame of this step, R - 1 (needed on rebase steps only)
        if (rebase) {
            float Rm[VN][DD];
            double kp[VN][DD];
#pragma unroll
            for (int c = 0; c < DD; ++c) {
                const VF v = *reinterpret_cast<const VF*>(a.Rm + c * Np + n0);
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    Rm[j][c] = v.v[j];
                    kp[j][c] = kprev[c * Np + n0 + j];
                }
            }
#pragma unroll
            for (int j = 0; j < VN; ++j) frame_advance<D>(kp[j], Rm[j], F[j]);
        }
        float acc[VN][NS];
#pragma unroll
        for (int j = 0; j < VN; ++j)
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[j][i] = 0.0f;

        const int l0 = chunk * chunk_len;
        const int l1 = min(L, l0 + chunk_len);
        // the packed words of one slot: exponent bytes and mantissa words of Q - 1 and kappa.  The next
        // slot's words are loaded before this slot is decoded (one slot of loads always in flight).  No
        // branch on empty or retired slots: they have weight 0 and hold finite data from their last use,
        // so they add exactly 0.
        struct Packed { unsigned qe, ke; VW qv[DD], kv[DD]; };
        auto load_packed = [&](int l, Packed& pk) {
            pk.qe = VN == 4 ? *reinterpret_cast<const unsigned*>(a.Qe + (long long)l * Np + n0)
                            : *reinterpret_cast<const unsigned short*>(a.Qe + (long long)l * Np + n0);
            pk.ke = VN == 4 ? *reinterpret_cast<const unsigned*>(a.Ke + (long long)l * Np + n0)
                            : *reinterpret_cast<const unsigned short*>(a.Ke + (long long)l * Np + n0);
#pragma unroll
            for (int c = 0; c < DD; ++c) {
                pk.qv[c] = *reinterpret_cast<const VW*>(a.Qm + ((long long)l * DD + c) * Np + n0);
                pk.kv[c] = *reinterpret_cast<const VW*>(a.Km + ((long long)l * DD + c) * Np + n0);
            }
        };
        Packed nxt;
        if (l0 < l1) load_packed(l0, nxt);
        for (int l = l0; l < l1; ++l) {
            const Packed cur = nxt;
            if (l + 1 < l1) load_packed(l + 1, nxt);
            const float w = s_w[l];
            float kap[VN][DD], Qd[VN][DD];
            {
                S16Scale sq[VN], sk[VN];
#pragma unroll
                for (int j = 0; j < VN; ++j) { sq[j] = S16Scale(s16_exp(cur.qe, j)); sk[j] = S16Scale(s16_exp(cur.ke, j)); }
#pragma unroll
                for (int c = 0; c < DD; ++c) {
#pragma unroll
                    for (int p2 = 0; p2 < VN / 2; ++p2) {
                        Qd[2 * p2][c] = s16_lo(cur.qv[c].v[p2], sq[2 * p2]);
                        Qd[2 * p2 + 1][c] = s16_hi(cur.qv[c].v[p2], sq[2 * p2 + 1]);
                        kap[2 * p2][c] = s16_lo(cur.kv[c].v[p2], sk[2 * p2]);
                        kap[2 * p2 + 1][c] = s16_hi(cur.kv[c].v[p2], sk[2 * p2 + 1]);
                    }
                }
            }
            const int part = s_part[l];
            if (part >= 0) {   // older half of a merge: kappa averaged with the newer half
                const unsigned ke2 = VN == 4 ? *reinterpret_cast<const unsigned*>(a.Ke + (long long)part * Np + n0)
                                             : *reinterpret_cast<const unsigned short*>(a.Ke + (long long)part * Np + n0);
                S16Scale sk2[VN];
#pragma unroll
                for (int j = 0; j < VN; ++j) sk2[j] = S16Scale(s16_exp(ke2, j));
#pragma unroll
                for (int c = 0; c < DD; ++c) {
                    const VW kv = *reinterpret_cast<const VW*>(a.Km + ((long long)part * DD + c) * Np + n0);
#pragma unroll
                    for (int p2 = 0; p2 < VN / 2; ++p2) {
                        kap[2 * p2][c] = 0.5f * (kap[2 * p2][c] + s16_lo(kv.v[p2], sk2[2 * p2]));
                        kap[2 * p2 + 1][c] = 0.5f * (kap[2 * p2 + 1][c] + s16_hi(kv.v[p2], sk2[2 * p2 + 1]));
                    }
                }
            }
            const float age = s_age[l];
#pragma unroll
            for (int j = 0; j < VN; ++j) point_integrand<D>(Qd[j], kap[j], age, w, inv_tau[j], inv_gc[j], acc[j]);
            if (rebase) {   // the point's Q becomes E(t, t') = R Q; the frame restarts at 1 in the commit
                unsigned short qm[VN][DD];
                VE qe_new;
#pragma unroll
                for (int j = 0; j < VN; ++j) {
                    float X[DD];
#pragma unroll
                    for (int r = 0; r < D; ++r)
#pragma unroll
                        for (int c = 0; c < D; ++c) {
                            float sum = F[j][r * D + c] + Qd[j][r * D + c];
#pragma unroll
                            for (int k = 0; k < D; ++k) sum += F[j][r * D + k] * Qd[j][k * D + c];
                            X[r * D + c] = sum;
                        }
                    unsigned char e;
                    s16_encode<DD>(X, qm[j], &e);
                    qe_new.v[j] = e;
                }
                *reinterpret_cast<VE*>(a.Qe + (long long)l * Np + n0) = qe_new;
#pragma unroll
                for (int c = 0; c < DD; ++c) {
                    VS qv;
#pragma unroll
                    for (int j = 0; j < VN; ++j) qv.v[j] = qm[j][c];
                    *reinterpret_cast<VS*>(a.Qm + ((long long)l * DD + c) * Np + n0) = qv;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            VF v;
#pragma unroll
            for (int j = 0; j < VN; ++j) v.v[j] = acc[j][i];
            *reinterpret_cast<VF*>(const_cast<float*>(a.part) + ((long long)chunk * NS + i) * Np + n0) = v;
        }
    }
}

// Commit alone (history-only test hook): the gradient comes from the caller.
template <int D, class H>
__global__ void __launch_bounds__(256) k_commit(H a, const double* __restrict__ kappa_in,
                                                double* __restrict__ sigma_f, double* __restrict__ kappa_f,
                                                double* __restrict__ sigma_out, const long long* t_dev, Geom g) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    __shared__ BlockStep s_bs[LBVE_MAXB];
    const long long t = *t_dev;
    sched_step_cta(a.B, a.C, t, s_bs);
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    double ktd[DD], kprev[DD], sig[NS];
#pragma unroll
    for (int c = 0; c < DD; ++c) {
        ktd[c] = kappa_in[(long long)c * g.N + n];
        kprev[c] = kappa_f[c * g.Npad + n];
    }
    hist_commit_any<D>(Arith<double>(), a, s_bs, g.Npad, n, kprev, ktd, g.ch[chan_index(g, n)], sig, t);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        sigma_f[i * g.Npad + n] = sig[i];
        sigma_out[(long long)i * g.N + n] = sig[i];
    }
#pragma unroll
    for (int c = 0; c < DD; ++c) kappa_f[c * g.Npad + n] = ktd[c];
}

}  // namespace lbk
