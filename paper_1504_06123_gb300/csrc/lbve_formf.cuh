// lbve_formf.cuh -- history form F: the paper's factor storage (Sec. III, Eq. eeval), on the GPU.
//
// Every retained point keeps, written once, its factor deviation Y = F - 1 -- F = exp(kappa(t') dt) for the
// point created at t', and for a merged point the product of the two merged factors, newer on the left --
// and its rate of strain Dm = kappa(t') + kappa(t')^T (packed symmetric; the averaged rate for a merged
// point).  Nothing per point is rewritten afterwards: every step re-forms E(t, t'_k) = F_1 F_2 ... F_k as the
// ordered product of the factors of all points from the newest to point k (Eq. eeval), which is what the
// paper's scheme does.  Dm alone carries what the integrand needs of kappa(t'): -d_t'B = E Dm E^T and
// gammadot(t')^2 = (1/2) tr Dm^2 (Sec. II).
//
// Sweep (k_sweep_f, k_sweep_f16): the points in memory are listed by age rank (newest first); a task takes
// one node tile and one contiguous range of ranks (a chunk) and forms the running product P = F_{r0} ... F_r
// of its own chunk, X = P - 1 carried in registers with the deviation product X <- X + Y + X Y, while it
// sums w G(t, t') (1 + X) Dm (1 + X)^T.  The chunk before it contributes the carry C_j = T_1 ... T_{j-1} of
// the chunks' total products T, so that E = C_j (1 + X): the chunk writes its local sum M_j and its product
// deviation T_j - 1, and the commit adds C_j M_j C_j^T over the chunks in order (the carry leaves the point
// sum like a frame: every point of the chunk sees the same C_j).  One read-only pass over the history.
//
// Commit (per node, fused into the collide kernel): sigma_struc(t) from the chunk records plus the point
// created now (age 0, E = 1, weight 1/2), then the block merges of the quasi-logarithmic grid (older point's
// time, factor product F_newer F_older, averaged Dm) and the new point (its factor exp(kappa(t)), formed in
// double and rounded once to the storage).
//
// Storage: float or double planes, or 16-bit block-scaled (d*d int16 mantissas of Y and NS of Dm, one shared
// power-of-two exponent byte per vector, as in the reduced-precision history of lbve_kernels.cuh).
#pragma once
#include "lbve_kernels.cuh"

namespace lbk {

// Packed symmetric components: xx, yy, xy (2D); xx, yy, zz, xy, xz, yz (3D).
template <int D> __host__ __device__ __forceinline__ constexpr int symr(int i) { return D == 2 ? (i == 1 ? 1 : 0) : (i < 3 ? i : (i == 5 ? 1 : 0)); }
template <int D> __host__ __device__ __forceinline__ constexpr int symc(int i) { return D == 2 ? (i == 0 ? 0 : 1) : (i < 3 ? i : (i == 3 ? 1 : 2)); }
template <int D> __host__ __device__ __forceinline__ constexpr int symi(int r, int c) {
    return D == 2 ? (r == c ? r : 2) : (r == c ? r : (r + c == 1 ? 3 : (r + c == 2 ? 4 : 5)));
}

// The modulus of Eq. (nlmax) (without G_inf) times the trapezoidal weight, per point.
// float: exp(-age (1/tau + gammadot/gamma_c)) = 2^(age (c1 + gammadot c2)) with c1 = -log2(e)/tau and
// c2 = -log2(e)/gamma_c folded per node, on the hardware exp2 and sqrt approximations (relative error about
// 2^-22); double: the library exp and sqrt.
template <typename R> struct PtMath;
template <> struct PtMath<float> {
    __device__ static __forceinline__ void consts(double inv_tau, double inv_gc, float& c1, float& c2) {
        c1 = (float)(-1.4426950408889634 * inv_tau);
        c2 = (float)(-1.4426950408889634 * inv_gc);
    }
    __device__ static __forceinline__ float sqrt_pos(float x) {
        float y;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static __forceinline__ float gw(float w, float age, float c1, float c2, float gd) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(age * fmaf(gd, c2, c1)));
        return w * y;
    }
};
template <> struct PtMath<double> {
    __device__ static __forceinline__ void consts(double inv_tau, double inv_gc, double& c1, double& c2) {
        c1 = inv_tau;
        c2 = inv_gc;
    }
    __device__ static __forceinline__ double sqrt_pos(double x) { return ::sqrt(x); }
    __device__ static __forceinline__ double gw(double w, double age, double c1, double c2, double gd) {
        return w * ::exp(-(age * (c1 + gd * c2)));
    }
};

// w G (1 + X) Dm (1 + X)^T added to acc (packed symmetric), Dm packed symmetric:
// F = Dm + X Dm, then the upper triangle of F (1 + X)^T = F + F X^T; gammadot^2 = (1/2) tr Dm^2.
template <int D, typename R>
__device__ __forceinline__ void sym_integrand(const R* X, const R* Dp, R age, R w, R c1, R c2, R* acc) {
    constexpr int NS = D == 2 ? 3 : 6;
    R Dm[D * D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) Dm[r * D + c] = Dp[symi<D>(r, c)];
    R F[D * D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = Dm[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s = ::fma(X[r * D + k], Dm[k * D + c], s);
            F[r * D + c] = s;
        }
    R h = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) h = ::fma(Dp[i], (i < D ? R(0.5) : R(1)) * Dp[i], h);
    const R g = PtMath<R>::gw(w, age, c1, c2, PtMath<R>::sqrt_pos(h));
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int r = symr<D>(i), c = symc<D>(i);
        R s = F[r * D + c];
#pragma unroll
        for (int k = 0; k < D; ++k) s = ::fma(F[r * D + k], X[c * D + k], s);
        acc[i] = ::fma(g, s, acc[i]);
    }
}

// X <- X + Y + X Y: the running product P <- P F in deviation form (P = 1 + X, F = 1 + Y).
template <int D, typename R>
__device__ __forceinline__ void dev_product(R* X, const R* Y) {
    R Xn[D * D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = X[r * D + c] + Y[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s = ::fma(X[r * D + k], Y[k * D + c], s);
            Xn[r * D + c] = s;
        }
#pragma unroll
    for (int i = 0; i < D * D; ++i) X[i] = Xn[i];
}

// ------------------------------------------------------------------------------------------------
// Rank tables of the sweep (shared memory): the points in memory after step t-1 listed newest first --
// the finest block from its newest point back, then each coarser block -- with their slot, age, trapezoidal
// weight at step t and merge partner (the newer half whose Dm is averaged into the older one; -1 if none).
// ------------------------------------------------------------------------------------------------
__host__ __device__ inline size_t sweep_f_smem_bytes(int L) {
    return ((size_t)L * 16 + sizeof(BlockStep) * LBVE_MAXB + sizeof(int) * (LBVE_MAXB + 1) + 15) / 16 * 16;
}

struct RankTab {
    int* slot;
    float* age;
    float* w;
    int* partner;
    int n;            // points in memory
};

__device__ __forceinline__ RankTab rank_tables(unsigned char* smem, int B, int C, long long t) {
    const int L = B * C;
    RankTab rt;
    rt.slot = reinterpret_cast<int*>(smem);
    rt.age = reinterpret_cast<float*>(rt.slot + L);
    rt.w = rt.age + L;
    rt.partner = reinterpret_cast<int*>(rt.w + L);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(rt.partner + L);
    int* s_off = reinterpret_cast<int*>(s_bs + LBVE_MAXB);   // first rank of each block, then the total
    if (threadIdx.x == 0) {
        sched_step(B, C, t, s_bs);
        int r = 0;
        for (int bb = B - 1; bb >= 0; --bb) {
            s_off[bb] = r;
            r += s_bs[bb].count_prev;
        }
        s_off[LBVE_MAXB] = r;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const int bb = l / C, j = l - (l / C) * C;
        int k = s_bs[bb].head_prev - j;
        if (k < 0) k += C;
        if (k >= s_bs[bb].count_prev) continue;       // empty ring slot: not a point
        int age, part;
        const float w = sched_slot_role(s_bs, C, bb, j, &age, &part);
        const int r = s_off[bb] + k;
        rt.slot[r] = l;
        rt.age[r] = (float)age;
        rt.w[r] = w;
        rt.partner[r] = part;
    }
    __syncthreads();
    rt.n = s_off[LBVE_MAXB];
    return rt;
}

// ------------------------------------------------------------------------------------------------
// Form F, float or double planes
// ------------------------------------------------------------------------------------------------
template <typename R> struct CommitF {
    R* __restrict__ Y;          // [L][DD][Npad] factor deviation F - 1 of each point
    R* __restrict__ Dm;         // [L][NS][Npad] rate of strain kappa + kappa^T (packed symmetric)
    R* __restrict__ part;       // [S][NS + DD][Npad] per chunk: the sum M (NS) and the product deviation T - 1 (DD)
    int B, C, S;
};

template <int D, typename R, int VN>
__global__ void __launch_bounds__(256, 2) k_sweep_f(CommitF<R> a, const long long* __restrict__ t_dev, Geom g) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    using V = Vec<R, VN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long t = *t_dev;
    const RankTab rt = rank_tables(smem_raw, a.B, a.C, t);
    const long long Np = g.Npad;
    const int lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int tiles = (int)(Np / (32 * VN));
    const int tasks = tiles * a.S;
    const int chunk_len = (rt.n + a.S - 1) / a.S;

    for (int task = gwarp; task < tasks; task += nwarps) {
        const int tile = task % tiles;
        const int chunk = task / tiles;
        const long long n0 = (long long)tile * 32 * VN + lane * VN;
        R c1[VN], c2[VN];
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            const Chan& c = g.ch[chan_index(g, n0 + j)];
            PtMath<R>::consts(c.inv_tau, c.inv_gc, c1[j], c2[j]);
        }
        R X[VN][DD], acc[VN][NS];
#pragma unroll
        for (int j = 0; j < VN; ++j) {
#pragma unroll
            for (int i = 0; i < DD; ++i) X[j][i] = 0;
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[j][i] = 0;
        }
        const int r0 = min(rt.n, chunk * chunk_len), r1 = min(rt.n, r0 + chunk_len);
        struct Pt { V y[DD], d[NS]; };
        auto load = [&](int r, Pt& p) {
            const long long l = rt.slot[r];
#pragma unroll
            for (int c = 0; c < DD; ++c) p.y[c] = *reinterpret_cast<const V*>(a.Y + (l * DD + c) * Np + n0);
#pragma unroll
            for (int c = 0; c < NS; ++c) p.d[c] = *reinterpret_cast<const V*>(a.Dm + (l * NS + c) * Np + n0);
        };
        Pt nxt;
        if (r0 < r1) load(r0, nxt);
        for (int r = r0; r < r1; ++r) {
            const Pt cur = nxt;
            if (r + 1 < r1) load(r + 1, nxt);
            R Y[VN][DD], Dp[VN][NS];
#pragma unroll
            for (int j = 0; j < VN; ++j) {
#pragma unroll
                for (int c = 0; c < DD; ++c) Y[j][c] = cur.y[c].v[j];
#pragma unroll
                for (int c = 0; c < NS; ++c) Dp[j][c] = cur.d[c].v[j];
            }
            const int part = rt.partner[r];
            if (part >= 0) {   // older half of a merge: its rate of strain averaged with the newer half's
#pragma unroll
                for (int c = 0; c < NS; ++c) {
                    const V v = *reinterpret_cast<const V*>(a.Dm + ((long long)part * NS + c) * Np + n0);
#pragma unroll
                    for (int j = 0; j < VN; ++j) Dp[j][c] = R(0.5) * (Dp[j][c] + v.v[j]);
                }
            }
            const R age = (R)rt.age[r], w = (R)rt.w[r];
#pragma unroll
            for (int j = 0; j < VN; ++j) {
                dev_product<D>(X[j], Y[j]);
                sym_integrand<D>(X[j], Dp[j], age, w, c1[j], c2[j], acc[j]);
            }
        }
        R* out = a.part + (long long)chunk * (NS + DD) * Np + n0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            V v;
#pragma unroll
            for (int j = 0; j < VN; ++j) v.v[j] = acc[j][i];
            *reinterpret_cast<V*>(out + i * Np) = v;
        }
#pragma unroll
        for (int i = 0; i < DD; ++i) {
            V v;
#pragma unroll
            for (int j = 0; j < VN; ++j) v.v[j] = X[j][i];
            *reinterpret_cast<V*>(out + (NS + i) * Np) = v;
        }
    }
}

// sigma_struc of a node from the chunk records, in double: sum_j C_j M_j C_j^T with C_1 = 1 and
// C_{j+1} = C_j T_j, plus the point created now (E = 1, weight 1/2, G = G_inf: (1/2) Dm(t)).
template <int D, typename R>
__device__ __forceinline__ void formf_sigma(const R* part, int S, long long Np, int n, const double* dnew, double G_inf,
                                            double* sig) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    double Z[DD], acc[NS];
#pragma unroll
    for (int i = 0; i < DD; ++i) Z[i] = 0.0;
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i] = 0.0;
    for (int j = 0; j < S; ++j) {
        const R* pj = part + (long long)j * (NS + DD) * Np + n;
        double M[DD], T[DD];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const double v = (double)pj[i * Np];
            M[symr<D>(i) * D + symc<D>(i)] = v;
            M[symc<D>(i) * D + symr<D>(i)] = v;
        }
#pragma unroll
        for (int i = 0; i < DD; ++i) T[i] = (double)pj[(NS + i) * Np];
        // C M C^T with C = 1 + Z: (M + Z M) (1 + Z)^T, upper triangle
        double F[DD];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                double s = M[r * D + c];
#pragma unroll
                for (int k = 0; k < D; ++k) s += Z[r * D + k] * M[k * D + c];
                F[r * D + c] = s;
            }
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int r = symr<D>(i), c = symc<D>(i);
            double s = F[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s += F[r * D + k] * Z[c * D + k];
            acc[i] += s;
        }
        dev_product<D>(Z, T);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) sig[i] = G_inf * (acc[i] + 0.5 * dnew[i]);
}

// exp(kappa) - 1 of the new point's factor, in double (Taylor to 8th order: |kappa| <= 1e-2 leaves < 1e-20).
template <int D>
__device__ __forceinline__ void factor_dev(const double* ktd, double* Y) { expm1_mat<D, double>(ktd, Y); }

template <int D>
__device__ __forceinline__ void rate_of_strain(const double* ktd, double* dp) {
    constexpr int NS = D == 2 ? 3 : 6;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int r = symr<D>(i), c = symc<D>(i);
        dp[i] = ktd[r * D + c] + ktd[c * D + r];
    }
}

template <int D, typename R>
__device__ __forceinline__ void hist_commit_any(const CommitF<R>& a, const BlockStep* s_bs, long long Np, int n,
                                                const double* /*kprev*/, const double* ktd, const Chan& p,
                                                double* sig, long long /*t*/) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    // the new point's stored values (rounded to the storage), used for its own contribution as for any point
    double Yn[DD], dn[NS];
    factor_dev<D>(ktd, Yn);
    rate_of_strain<D>(ktd, dn);
#pragma unroll
    for (int i = 0; i < NS; ++i) dn[i] = (double)(R)dn[i];
    formf_sigma<D, R>(a.part, a.S, Np, n, dn, p.G_inf, sig);
    // block merges, coarsest first (every ring slot is read before it is overwritten): the older point's
    // time, the factor F_newer F_older, the average of the two rates
    for (int bb = 1; bb < a.B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long s1 = (long long)bb * a.C + o1, s2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
        double Y1[DD], Y2[DD];
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            Y1[c] = (double)a.Y[(s1 * DD + c) * Np + n];
            Y2[c] = (double)a.Y[(s2 * DD + c) * Np + n];
        }
        dev_product<D>(Y2, Y1);   // (1 + Y2)(1 + Y1) - 1
        double d1[NS], d2[NS];
#pragma unroll
        for (int c = 0; c < NS; ++c) {
            d1[c] = (double)a.Dm[(s1 * NS + c) * Np + n];
            d2[c] = (double)a.Dm[(s2 * NS + c) * Np + n];
        }
#pragma unroll
        for (int c = 0; c < DD; ++c) a.Y[(dst * DD + c) * Np + n] = (R)Y2[c];
#pragma unroll
        for (int c = 0; c < NS; ++c) a.Dm[(dst * NS + c) * Np + n] = (R)(0.5 * (d1[c] + d2[c]));
    }
    const long long dst = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
#pragma unroll
    for (int c = 0; c < DD; ++c) a.Y[(dst * DD + c) * Np + n] = (R)Yn[c];
#pragma unroll
    for (int c = 0; c < NS; ++c) a.Dm[(dst * NS + c) * Np + n] = (R)dn[c];
}

// ------------------------------------------------------------------------------------------------
// Form F, 16-bit block-scaled storage (the reduced-precision history): Y and Dm each as int16 mantissas
// sharing one power-of-two exponent byte (s16_encode / s16_decode of lbve_kernels.cuh); FP32 arithmetic.
// ------------------------------------------------------------------------------------------------
struct CommitF16 {
    unsigned short* __restrict__ Ym;  // [L][DD][Npad] biased mantissas of Y = F - 1
    unsigned char* __restrict__ Ye;   // [L][Npad] biased exponents
    unsigned short* __restrict__ Dmm; // [L][NS][Npad] biased mantissas of Dm
    unsigned char* __restrict__ De;   // [L][Npad]
    float* __restrict__ part;         // [S][NS + DD][Npad]
    int B, C, S;
};

template <int D, int VN>
__global__ void __launch_bounds__(256, 2) k_sweep_f16(CommitF16 a, const long long* __restrict__ t_dev, Geom g) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    static_assert(VN == 2 || VN == 4, "packed decode handles 2 or 4 nodes per lane");
    using VW = Vec<unsigned, VN / 2>;
    using VF = Vec<float, VN>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long t = *t_dev;
    const RankTab rt = rank_tables(smem_raw, a.B, a.C, t);
    const long long Np = g.Npad;
    const int lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int tiles = (int)(Np / (32 * VN));
    const int tasks = tiles * a.S;
    const int chunk_len = (rt.n + a.S - 1) / a.S;

    for (int task = gwarp; task < tasks; task += nwarps) {
        const int tile = task % tiles;
        const int chunk = task / tiles;
        const long long n0 = (long long)tile * 32 * VN + lane * VN;
        float c1[VN], c2[VN];
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            const Chan& c = g.ch[chan_index(g, n0 + j)];
            PtMath<float>::consts(c.inv_tau, c.inv_gc, c1[j], c2[j]);
        }
        float X[VN][DD], acc[VN][NS];
#pragma unroll
        for (int j = 0; j < VN; ++j) {
#pragma unroll
            for (int i = 0; i < DD; ++i) X[j][i] = 0.0f;
#pragma unroll
            for (int i = 0; i < NS; ++i) acc[j][i] = 0.0f;
        }
        const int r0 = min(rt.n, chunk * chunk_len), r1 = min(rt.n, r0 + chunk_len);
        struct Packed { unsigned ye, de; VW y[DD], d[NS]; };
        auto load_exp = [&](const unsigned char* base, long long l) -> unsigned {
            return VN == 4 ? *reinterpret_cast<const unsigned*>(base + l * Np + n0)
                           : *reinterpret_cast<const unsigned short*>(base + l * Np + n0);
        };
        auto load = [&](int r, Packed& p) {
            const long long l = rt.slot[r];
            p.ye = load_exp(a.Ye, l);
            p.de = load_exp(a.De, l);
#pragma unroll
            for (int c = 0; c < DD; ++c) p.y[c] = *reinterpret_cast<const VW*>(a.Ym + (l * DD + c) * Np + n0);
#pragma unroll
            for (int c = 0; c < NS; ++c) p.d[c] = *reinterpret_cast<const VW*>(a.Dmm + (l * NS + c) * Np + n0);
        };
        Packed nxt;
        if (r0 < r1) load(r0, nxt);
        for (int r = r0; r < r1; ++r) {
            const Packed cur = nxt;
            if (r + 1 < r1) load(r + 1, nxt);
            float Y[VN][DD], Dp[VN][NS];
            {
                S16Scale sy[VN], sd[VN];
#pragma unroll
                for (int j = 0; j < VN; ++j) { sy[j] = S16Scale(s16_exp(cur.ye, j)); sd[j] = S16Scale(s16_exp(cur.de, j)); }
#pragma unroll
                for (int p2 = 0; p2 < VN / 2; ++p2) {
#pragma unroll
                    for (int c = 0; c < DD; ++c) {
                        Y[2 * p2][c] = s16_lo(cur.y[c].v[p2], sy[2 * p2]);
                        Y[2 * p2 + 1][c] = s16_hi(cur.y[c].v[p2], sy[2 * p2 + 1]);
                    }
#pragma unroll
                    for (int c = 0; c < NS; ++c) {
                        Dp[2 * p2][c] = s16_lo(cur.d[c].v[p2], sd[2 * p2]);
                        Dp[2 * p2 + 1][c] = s16_hi(cur.d[c].v[p2], sd[2 * p2 + 1]);
                    }
                }
            }
            const int part = rt.partner[r];
            if (part >= 0) {   // older half of a merge: rate of strain averaged with the newer half's
                const unsigned de2 = load_exp(a.De, part);
                S16Scale s2[VN];
#pragma unroll
                for (int j = 0; j < VN; ++j) s2[j] = S16Scale(s16_exp(de2, j));
#pragma unroll
                for (int c = 0; c < NS; ++c) {
                    const VW v = *reinterpret_cast<const VW*>(a.Dmm + ((long long)part * NS + c) * Np + n0);
#pragma unroll
                    for (int p2 = 0; p2 < VN / 2; ++p2) {
                        Dp[2 * p2][c] = 0.5f * (Dp[2 * p2][c] + s16_lo(v.v[p2], s2[2 * p2]));
                        Dp[2 * p2 + 1][c] = 0.5f * (Dp[2 * p2 + 1][c] + s16_hi(v.v[p2], s2[2 * p2 + 1]));
                    }
                }
            }
            const float age = rt.age[r], w = rt.w[r];
#pragma unroll
            for (int j = 0; j < VN; ++j) {
                dev_product<D>(X[j], Y[j]);
                sym_integrand<D>(X[j], Dp[j], age, w, c1[j], c2[j], acc[j]);
            }
        }
        float* out = a.part + (long long)chunk * (NS + DD) * Np + n0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            VF v;
#pragma unroll
            for (int j = 0; j < VN; ++j) v.v[j] = acc[j][i];
            *reinterpret_cast<VF*>(out + i * Np) = v;
        }
#pragma unroll
        for (int i = 0; i < DD; ++i) {
            VF v;
#pragma unroll
            for (int j = 0; j < VN; ++j) v.v[j] = X[j][i];
            *reinterpret_cast<VF*>(out + (NS + i) * Np) = v;
        }
    }
}

// Block-scaled 16-bit encode / decode of one vector of M doubles (rounded through float).
template <int M>
__device__ __forceinline__ void f16_store(const double* v, unsigned short* m, unsigned char* e, long long stride, long long at) {
    float f[M];
    unsigned short u[M];
    unsigned char eb;
#pragma unroll
    for (int i = 0; i < M; ++i) f[i] = (float)v[i];
    s16_encode<M>(f, u, &eb);
#pragma unroll
    for (int i = 0; i < M; ++i) m[at + i * stride] = u[i];
    *e = eb;
}

template <int M>
__device__ __forceinline__ void f16_load(const unsigned short* m, unsigned char eb, long long stride, long long at, double* v) {
    unsigned short u[M];
    float f[M];
#pragma unroll
    for (int i = 0; i < M; ++i) u[i] = m[at + i * stride];
    s16_decode<M>(u, eb, f);
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = (double)f[i];
}

template <int D>
__device__ __forceinline__ void hist_commit_any(const CommitF16& a, const BlockStep* s_bs, long long Np, int n,
                                                const double* /*kprev*/, const double* ktd, const Chan& p,
                                                double* sig, long long /*t*/) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    double Yn[DD], dn[NS];
    factor_dev<D>(ktd, Yn);
    rate_of_strain<D>(ktd, dn);
    // the new point as stored: encoded once, its own contribution from the stored (rounded) rate
    const long long dst_new = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
    unsigned short um[NS];
    unsigned char ue;
    {
        float f[NS];
#pragma unroll
        for (int i = 0; i < NS; ++i) f[i] = (float)dn[i];
        s16_encode<NS>(f, um, &ue);
        s16_decode<NS>(um, ue, f);
#pragma unroll
        for (int i = 0; i < NS; ++i) dn[i] = (double)f[i];
    }
    formf_sigma<D, float>(a.part, a.S, Np, n, dn, p.G_inf, sig);
    for (int bb = 1; bb < a.B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long s1 = (long long)bb * a.C + o1, s2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
        double Y1[DD], Y2[DD], d1[NS], d2[NS];
        f16_load<DD>(a.Ym, a.Ye[s1 * Np + n], Np, s1 * DD * Np + n, Y1);
        f16_load<DD>(a.Ym, a.Ye[s2 * Np + n], Np, s2 * DD * Np + n, Y2);
        f16_load<NS>(a.Dmm, a.De[s1 * Np + n], Np, s1 * NS * Np + n, d1);
        f16_load<NS>(a.Dmm, a.De[s2 * Np + n], Np, s2 * NS * Np + n, d2);
        dev_product<D>(Y2, Y1);
#pragma unroll
        for (int c = 0; c < NS; ++c) d1[c] = 0.5 * (d1[c] + d2[c]);
        f16_store<DD>(Y2, a.Ym, a.Ye + dst * Np + n, Np, dst * DD * Np + n);
        f16_store<NS>(d1, a.Dmm, a.De + dst * Np + n, Np, dst * NS * Np + n);
    }
    f16_store<DD>(Yn, a.Ym, a.Ye + dst_new * Np + n, Np, dst_new * DD * Np + n);
#pragma unroll
    for (int i = 0; i < NS; ++i) a.Dmm[(dst_new * NS + i) * Np + n] = um[i];
    a.De[dst_new * Np + n] = ue;
}

}  // namespace lbk
