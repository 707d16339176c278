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
// sum like a frame: every point of the chunk sees the same C_j).  One read-only pass over the history.  The
// chunk holding the oldest point needs no T (nothing follows it); the 16-bit sweep sums that chunk in
// Horner form from its oldest point to its newest, H <- F (H + w G Dm) F^T, one congruence per point in
// place of the running product and the sandwich (the same sum, the additions in another order).
//
// Commit (per node, fused into the collide kernel): sigma_struc(t) from the chunk records plus the point
// created now (age 0, E = 1, weight 1/2), then the block merges of the quasi-logarithmic grid (older point's
// time, factor product F_newer F_older, averaged Dm) and the new point (its factor exp(kappa(t))), all in the
// history's arithmetic (float for the FP32 and 16-bit storages, double for FP64), each chunk's stress term
// added in double.
//
// Storage: float or double planes, or 16-bit block-scaled (d*d int16 mantissas of Y and NS of Dm, one shared
// power-of-two exponent byte per vector, as in the reduced-precision history of lbve_kernels.cuh).
#pragma once
#include <type_traits>

#include "lbve_kernels.cuh"

namespace lbk {

// Packed symmetric components: xx, yy, xy (2D); xx, yy, zz, xy, xz, yz (3D).
template <int D> __host__ __device__ __forceinline__ constexpr int symr(int i) { return D == 2 ? (i == 1 ? 1 : 0) : (i < 3 ? i : (i == 5 ? 1 : 0)); }
template <int D> __host__ __device__ __forceinline__ constexpr int symc(int i) { return D == 2 ? (i == 0 ? 0 : 1) : (i < 3 ? i : (i == 3 ? 1 : 2)); }
template <int D> __host__ __device__ __forceinline__ constexpr int symi(int r, int c) {
    return D == 2 ? (r == c ? r : 2) : (r == c ? r : (r + c == 1 ? 3 : (r + c == 2 ? 4 : 5)));
}

// The modulus of Eq. (nlmax) (without G_inf) times the trapezoidal weight, per point.
// float: w exp(-age (1/tau + gammadot/gamma_c)) = 2^(age (c1 + gammadot c2) + log2 w) with c1 = -log2(e)/tau
// and c2 = -log2(e)/gamma_c folded per node and log2 w per rank (the argument wx), on the hardware exp2 and
// sqrt approximations (relative error about 2^-22); double: wx = w and the library exp and sqrt.
template <typename R> struct PtMath;
template <> struct PtMath<float> {
    static constexpr bool kLog2W = true;
    __device__ static __forceinline__ void consts(double inv_tau, double inv_gc, float& c1, float& c2) {
        c1 = (float)(-1.4426950408889634 * inv_tau);
        c2 = (float)(-1.4426950408889634 * inv_gc);
    }
    __device__ static __forceinline__ float sqrt_pos(float x) {
        float y;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    __device__ static __forceinline__ float gw(float lw, float age, float c1, float c2, float gd) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fmaf(age, fmaf(gd, c2, c1), lw)));
        return y;
    }
};
template <> struct PtMath<double> {
    static constexpr bool kLog2W = false;
    __device__ static __forceinline__ void consts(double inv_tau, double inv_gc, double& c1, double& c2) {
        c1 = inv_tau;
        c2 = inv_gc;
    }
    __device__ static __forceinline__ double sqrt_pos(double x) { return ::sqrt(x); }
    __device__ static __forceinline__ double gw(double w, double age, double c1, double c2, double gd) {
        return w * ::exp(-(age * (c1 + gd * c2)));
    }
};

// w G of one point: gammadot^2 = (1/2) tr Dm^2 from the packed Dm, then the modulus and weight as one exp.
template <int D, typename R>
__device__ __forceinline__ R point_weight(const R* Dp, R age, R w, R c1, R c2) {
    constexpr int NS = D == 2 ? 3 : 6;
    R h = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) h = ::fma(Dp[i], (i < D ? R(0.5) : R(1)) * Dp[i], h);
    return PtMath<R>::gw(w, age, c1, c2, PtMath<R>::sqrt_pos(h));
}

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
    const R g = point_weight<D>(Dp, age, w, c1, c2);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int r = symr<D>(i), c = symc<D>(i);
        R s = F[r * D + c];
#pragma unroll
        for (int k = 0; k < D; ++k) s = ::fma(F[r * D + k], X[c * D + k], s);
        acc[i] = ::fma(g, s, acc[i]);
    }
}

// H <- (1 + Y) H (1 + Y)^T, H packed symmetric: G = H + Y H, then the upper triangle of G (1 + Y)^T = G + G Y^T.
// One step of the Horner form of a chunk's sum, taken from its oldest rank k = K to its newest k = 1:
// H_K = F_K (w_K G_K Dm_K) F_K^T, H_k = F_k (w_k G_k Dm_k + H_{k+1}) F_k^T, so that H_1 is the sum over k of
// w_k G_k P_k Dm_k P_k^T with P_k = F_1 ... F_k -- the chunk's M without forming P_k itself.
template <int D, typename R>
__device__ __forceinline__ void sym_congruence(R* H, const R* Y) {
    constexpr int NS = D == 2 ? 3 : 6;
    R Hm[D * D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) Hm[r * D + c] = H[symi<D>(r, c)];
    R G[D * D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            R s = Hm[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s = ::fma(Y[r * D + k], Hm[k * D + c], s);
            G[r * D + c] = s;
        }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int r = symr<D>(i), c = symc<D>(i);
        R s = G[r * D + c];
#pragma unroll
        for (int k = 0; k < D; ++k) s = ::fma(G[r * D + k], Y[c * D + k], s);
        H[i] = s;
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
// Rank table of the sweep (shared memory, one 16-byte entry per rank): the points in memory after step
// t-1 listed newest first -- the finest block from its newest point back, then each coarser block -- with
// their slot, merge partner (the newer half whose Dm is averaged into the older one; -1 if none), age and
// trapezoidal weight at step t.  LOG2W: the weight is stored as log2(w) (-inf for w = 0), for the float
// kernels that form w G as one exp2.
// ------------------------------------------------------------------------------------------------
__host__ __device__ inline size_t sweep_f_smem_bytes(int L) {
    return ((size_t)L * 16 + sizeof(BlockStep) * LBVE_MAXB + sizeof(int) * (LBVE_MAXB + 1) + 15) / 16 * 16;
}

struct RankEnt { int slot, partner; float age, w; };

struct RankTab {
    const RankEnt* e;
    int n;            // points in memory
};

template <bool LOG2W>
__device__ __forceinline__ RankTab rank_tables(unsigned char* smem, int B, int C, long long t) {
    const int L = B * C;
    RankEnt* ent = reinterpret_cast<RankEnt*>(smem);
    BlockStep* s_bs = reinterpret_cast<BlockStep*>(ent + L);
    int* s_off = reinterpret_cast<int*>(s_bs + LBVE_MAXB);   // first rank of each block, then the total
    sched_step_cta(B, C, t, s_bs);
    __syncthreads();
    if (threadIdx.x == 0) {
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
        RankEnt e;
        e.slot = l;
        e.partner = part;
        e.age = (float)age;
        e.w = LOG2W ? (w > 0.0f ? log2f(w) : -INFINITY) : w;
        ent[s_off[bb] + k] = e;
    }
    __syncthreads();
    RankTab rt;
    rt.e = ent;
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
    const RankTab rt = rank_tables<PtMath<R>::kLog2W>(smem_raw, a.B, a.C, t);
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
            const long long l = rt.e[r].slot;
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
            const RankEnt e = rt.e[r];
            R Y[VN][DD], Dp[VN][NS];
#pragma unroll
            for (int j = 0; j < VN; ++j) {
#pragma unroll
                for (int c = 0; c < DD; ++c) Y[j][c] = cur.y[c].v[j];
#pragma unroll
                for (int c = 0; c < NS; ++c) Dp[j][c] = cur.d[c].v[j];
            }
            if (e.partner >= 0) {   // older half of a merge: its rate of strain averaged with the newer half's
#pragma unroll
                for (int c = 0; c < NS; ++c) {
                    const V v = *reinterpret_cast<const V*>(a.Dm + ((long long)e.partner * NS + c) * Np + n0);
#pragma unroll
                    for (int j = 0; j < VN; ++j) Dp[j][c] = R(0.5) * (Dp[j][c] + v.v[j]);
                }
            }
            const R age = (R)e.age, w = (R)e.w;
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

// sigma_struc of a node from the chunk records: sum_j C_j M_j C_j^T with C_1 = 1 and C_{j+1} = C_j T_j (formed
// in the history's arithmetic A, each chunk's term added in the node arithmetic N), plus the point created
// now (E = 1, weight 1/2, G = G_inf: (1/2) Dm(t)).
template <int D, typename A, typename R, typename N>
__device__ __forceinline__ void formf_sigma(const R* part, int S, long long Np, int n, const N* dnew, N G_inf,
                                            N* sig) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    A Z[DD];
    N acc[NS];
#pragma unroll
    for (int i = 0; i < DD; ++i) Z[i] = A(0);
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i] = N(0);
#pragma unroll 4
    for (int j = 0; j < S; ++j) {
        const R* pj = part + (long long)j * (NS + DD) * Np + n;
        A M[DD], T[DD];
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const A v = (A)pj[i * Np];
            M[symr<D>(i) * D + symc<D>(i)] = v;
            M[symc<D>(i) * D + symr<D>(i)] = v;
        }
        // the last chunk's product is composed into nothing: not read (the 16-bit sweep does not write it)
        if (j + 1 < S) {
#pragma unroll
            for (int i = 0; i < DD; ++i) T[i] = (A)pj[(NS + i) * Np];
        }
        // C M C^T with C = 1 + Z: (M + Z M) (1 + Z)^T, upper triangle
        A F[DD];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                A s = M[r * D + c];
#pragma unroll
                for (int k = 0; k < D; ++k) s = ::fma(Z[r * D + k], M[k * D + c], s);
                F[r * D + c] = s;
            }
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int r = symr<D>(i), c = symc<D>(i);
            A s = F[r * D + c];
#pragma unroll
            for (int k = 0; k < D; ++k) s = ::fma(F[r * D + k], Z[c * D + k], s);
            acc[i] += (N)s;
        }
        if (j + 1 < S) dev_product<D>(Z, T);
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) sig[i] = G_inf * (acc[i] + N(0.5) * dnew[i]);
}

// exp(kappa) - 1 of the new point's factor in the arithmetic A (Taylor to 4th order in float, 8th in double:
// |kappa| <= 1e-2 leaves below 1e-12 and 1e-20).
template <int D, typename A, typename K>
__device__ __forceinline__ void factor_dev(const K* ktd, A* Y) {
    A k[D * D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) k[i] = (A)ktd[i];
    expm1_mat<D, A>(k, Y);
}

template <int D, typename K>
__device__ __forceinline__ void rate_of_strain(const K* ktd, K* dp) {
    constexpr int NS = D == 2 ? 3 : 6;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int r = symr<D>(i), c = symc<D>(i);
        dp[i] = ktd[r * D + c] + ktd[c * D + r];
    }
}

template <int D, typename R, typename N>
__device__ __forceinline__ void hist_commit_any(Arith<N>, const CommitF<R>& a, const BlockStep* s_bs, long long Np,
                                                int n, const double* /*kprev*/, const double* ktd, const Chan& p,
                                                N* sig, long long /*t*/) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    // the new point's stored values (rounded to the storage), used for its own contribution as for any point
    R Yn[DD];
    double dd[NS];
    N dn[NS];
    factor_dev<D, R>(ktd, Yn);
    rate_of_strain<D>(ktd, dd);
#pragma unroll
    for (int i = 0; i < NS; ++i) dn[i] = (N)(R)dd[i];
    formf_sigma<D, R, R, N>(a.part, a.S, Np, n, dn, chan_val<N>(p.G_inf, p.G_inf_f), sig);
    // block merges, coarsest first (every ring slot is read before it is overwritten): the older point's
    // time, the factor F_newer F_older, the average of the two rates
    for (int bb = 1; bb < a.B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long s1 = (long long)bb * a.C + o1, s2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
        R Y1[DD], Y2[DD];
#pragma unroll
        for (int c = 0; c < DD; ++c) {
            Y1[c] = a.Y[(s1 * DD + c) * Np + n];
            Y2[c] = a.Y[(s2 * DD + c) * Np + n];
        }
        dev_product<D>(Y2, Y1);   // (1 + Y2)(1 + Y1) - 1
#pragma unroll
        for (int c = 0; c < NS; ++c)
            a.Dm[(dst * NS + c) * Np + n] = R(0.5) * (a.Dm[(s1 * NS + c) * Np + n] + a.Dm[(s2 * NS + c) * Np + n]);
#pragma unroll
        for (int c = 0; c < DD; ++c) a.Y[(dst * DD + c) * Np + n] = Y2[c];
    }
    const long long dst = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
#pragma unroll
    for (int c = 0; c < DD; ++c) a.Y[(dst * DD + c) * Np + n] = Yn[c];
#pragma unroll
    for (int c = 0; c < NS; ++c) a.Dm[(dst * NS + c) * Np + n] = (R)dd[c];
}

// ------------------------------------------------------------------------------------------------
// Form F, 16-bit block-scaled storage (the reduced-precision history): Y and Dm each as int16 mantissas
// sharing one power-of-two exponent byte per vector (s16_encode / s16_decode of lbve_kernels.cuh); FP32
// arithmetic.
//
// Layout: node tiles of TN = 32 VN nodes (VN = 4 in 2D, 2 in 3D: one sweep lane's nodes); each (tile, slot)
// is one 2048-byte block, blocks ordered [tile][slot].  Inside a block, the 64 bytes of lane q (its VN
// nodes' 7 / 15 mantissas and their exponent bytes, as 32 half-words h) lie in four 16-byte pieces, piece k
// at byte k*512 + q*16: a warp reads one slot of its tile with four fully coalesced 16-byte loads per lane at
// fixed offsets, and a whole slot of a tile is one contiguous block.
//   2D: h = 4c + j  Y comp c (0..3) of node j;  h = 16 + 4c + j  Dm comp c (0..2);  h 28-29: the 4 Y exponent
//       bytes (node j in byte j);  h 30-31: the 4 Dm exponent bytes.
//   3D: h = 2c + j  Y comp c (0..8);  h = 18 + 2c + j  Dm comp c (0..5);  h 30: Y exponent bytes of the two
//       nodes;  h 31: Dm exponent bytes.
// ------------------------------------------------------------------------------------------------
template <int D> struct F16Layout {
    static constexpr int VN = D == 2 ? 4 : 2;       // nodes per lane
    static constexpr int TN = 32 * VN;              // nodes per tile
    static constexpr int DD = D * D, NS = D == 2 ? 3 : 6;
    static constexpr int kBlock = 2048;             // bytes per (tile, slot)
    __host__ __device__ static constexpr int y_half(int c, int j) { return c * VN + j; }
    __host__ __device__ static constexpr int d_half(int c, int j) { return DD * VN + c * VN + j; }
    __host__ __device__ static constexpr int ye_byte(int j) { return D == 2 ? 56 + j : 60 + j; }     // byte inside the lane's 64
    __host__ __device__ static constexpr int de_byte(int j) { return D == 2 ? 60 + j : 62 + j; }
    // byte offset of byte b (0..63) of lane q inside a block
    __host__ __device__ static constexpr int lane_byte(int q, int b) { return (b >> 4) * 512 + q * 16 + (b & 15); }
};

struct CommitF16 {
    unsigned char* __restrict__ blk;  // [tiles][L][2048] history blocks
    float* __restrict__ part;         // [S][NS + DD][Npad]
    int B, C, S;
    int bal_nw;                       // 0: chunk tasks (S chunks per tile); > 0: balanced ranges over bal_nw warps
};
template <> struct Hist16<CommitF16> { static constexpr bool value = true; };

// Balanced ranges of the 16-bit form-F sweep: with n points per node and `tiles` node tiles, warp w of nw
// takes the ranks [w Wp, (w + 1) Wp) of the tile-major sequence of (tile, rank), Wp = ceil(tiles n / nw), so
// every warp streams the same number of blocks.  A tile is cut at the multiples of Wp inside it; its
// pieces, in rank order, are owned by warps floor(t n / Wp) ... floor(((t + 1) n - 1) / Wp), and piece j
// writes chunk record j.  At most ceil(nw / tiles) + 1 pieces per tile.
__host__ __device__ inline long long f16_bal_wp(long long tiles, int n, int nw) { return (tiles * n + nw - 1) / nw; }
__host__ __device__ inline int f16_bal_pieces(long long tile, int n, long long wp) {
    return (int)(((tile + 1) * n - 1) / wp - (tile * n) / wp + 1);
}
__host__ __device__ inline int f16_bal_max_pieces(long long tiles, int nw) { return (int)((nw + tiles - 1) / tiles) + 1; }

// Ranks ahead of the one in process whose blocks a warp asks the L2 to fetch (one bulk prefetch of 2048 bytes
// per slot, issued by lane 0): the loads of those slots then hit the L2, and the DRAM requests in flight per
// warp are not bounded by the two register buffers.
#ifndef LBVE_F16_PREFETCH
#define LBVE_F16_PREFETCH 4
#endif

// Bulk prefetch of [p, p + bytes) into the L2 (p and bytes multiples of 16; no completion to wait for).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// One piece of work of the 16-bit form-F sweep: ranks [r0, r1) of tile `tile`, its sums (and product
// deviation) into chunk record `chunk`.  HZ: the tile's oldest piece (r1 = n), whose product the commit never
// composes -- summed in Horner form from its oldest rank to its newest (sym_congruence), one congruence per
// point instead of the running product plus the sandwich; other pieces run newest first with the running
// product.  The kernel calls each path from a loop of its own: one loop holding both spills registers.
template <int D, int VN, bool HZ>
__device__ __forceinline__ void f16_piece(const CommitF16 a, const RankEnt* __restrict__ ent, const int n_pts,
                                       const Geom g, const int tile, const int r0, const int r1, const int chunk) {
    using Lay = F16Layout<D>;
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    using VF = Vec<float, VN>;
    const RankTab rt{ent, n_pts};
    const long long Np = g.Npad;
    const int L = a.B * a.C;
    const int lane = threadIdx.x & 31;
    const long long n0 = (long long)tile * Lay::TN + lane * VN;
    const unsigned char* tbase = a.blk + (long long)tile * L * Lay::kBlock + lane * 16;
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
    const int m = r1 - r0;
    // rank of the q-th point visited
    auto rank_at = [&](int q) { return HZ ? r1 - 1 - q : r0 + q; };
    // the lane's 64 bytes of one slot as 16 words (word q holds half-words 2q, 2q + 1)
    auto load = [&](int q, unsigned (&wd)[16]) {
        const uint4* p = reinterpret_cast<const uint4*>(tbase + (long long)rt.e[rank_at(q)].slot * Lay::kBlock);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 v = p[k * 32];          // + k * 512 bytes
            wd[4 * k] = v.x; wd[4 * k + 1] = v.y; wd[4 * k + 2] = v.z; wd[4 * k + 3] = v.w;
        }
    };
    auto half_of = [&](const unsigned (&wd)[16], int h, const S16Scale& sc) -> float {
        return (h & 1) ? s16_hi(wd[h >> 1], sc) : s16_lo(wd[h >> 1], sc);
    };
    auto process = [&](int q, const unsigned (&wd)[16]) {
        const RankEnt e = rt.e[rank_at(q)];
        const unsigned ye = D == 2 ? wd[14] : (wd[15] & 0xFFFFu);
        const unsigned de = D == 2 ? wd[15] : (wd[15] >> 16);
        float Y[VN][DD], Dp[VN][NS];
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            const S16Scale sy(s16_exp(ye, j)), sd(s16_exp(de, j));
#pragma unroll
            for (int c = 0; c < DD; ++c) Y[j][c] = half_of(wd, Lay::y_half(c, j), sy);
#pragma unroll
            for (int c = 0; c < NS; ++c) Dp[j][c] = half_of(wd, Lay::d_half(c, j), sd);
        }
        if (e.partner >= 0) {   // older half of a merge: rate of strain averaged with the newer half's
            unsigned pw[16];
            {
                const uint4* p = reinterpret_cast<const uint4*>(tbase + (long long)e.partner * Lay::kBlock);
#pragma unroll
                for (int k = 2; k < 4; ++k) {   // the Dm mantissas and the exponents sit in pieces 2 and 3
                    const uint4 v = p[k * 32];
                    pw[4 * k] = v.x; pw[4 * k + 1] = v.y; pw[4 * k + 2] = v.z; pw[4 * k + 3] = v.w;
                }
            }
            const unsigned de2 = D == 2 ? pw[15] : (pw[15] >> 16);
#pragma unroll
            for (int j = 0; j < VN; ++j) {
                const S16Scale s2(s16_exp(de2, j));
#pragma unroll
                for (int c = 0; c < NS; ++c) Dp[j][c] = 0.5f * (Dp[j][c] + half_of(pw, Lay::d_half(c, j), s2));
            }
        }
#pragma unroll
        for (int j = 0; j < VN; ++j) {
            if (HZ) {
                const float wg = point_weight<D>(Dp[j], e.age, e.w, c1[j], c2[j]);
#pragma unroll
                for (int i = 0; i < NS; ++i) acc[j][i] = fmaf(wg, Dp[j][i], acc[j][i]);
                sym_congruence<D>(acc[j], Y[j]);
            } else {
                dev_product<D>(X[j], Y[j]);
                sym_integrand<D>(X[j], Dp[j], e.age, e.w, c1[j], c2[j], acc[j]);
            }
        }
    };
    // two slots of words alternate: the next slot's loads are in flight while a slot is processed; the
    // blocks of the points LBVE_F16_PREFETCH ahead in the visiting order are on their way to the L2
    constexpr int PF = LBVE_F16_PREFETCH;
    auto prefetch = [&](int q) {
        if (PF > 0 && lane == 0 && q < m) prefetch_l2_bulk(tbase + (long long)rt.e[rank_at(q)].slot * Lay::kBlock, Lay::kBlock);
    };
    for (int k = 2; k < PF; ++k) prefetch(k);
    unsigned wa[16], wb[16];
    if (m > 0) load(0, wa);
    for (int q = 0; q < m; q += 2) {
        if (q + 1 < m) load(q + 1, wb);
        prefetch(q + PF);
        process(q, wa);
        if (q + 1 >= m) break;
        if (q + 2 < m) load(q + 2, wa);
        prefetch(q + 1 + PF);
        process(q + 1, wb);
    }
    float* out = a.part + (long long)chunk * (NS + DD) * Np + n0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        VF v;
#pragma unroll
        for (int j = 0; j < VN; ++j) v.v[j] = acc[j][i];
        *reinterpret_cast<VF*>(out + i * Np) = v;
    }
    if (!HZ) {
#pragma unroll
        for (int i = 0; i < DD; ++i) {
            VF v;
#pragma unroll
            for (int j = 0; j < VN; ++j) v.v[j] = X[j][i];
            *reinterpret_cast<VF*>(out + (NS + i) * Np) = v;
        }
    }
}

template <int D, int VN>
__global__ void __launch_bounds__(256, 2) k_sweep_f16(CommitF16 a, const long long* __restrict__ t_dev, Geom g) {
    using Lay = F16Layout<D>;
    static_assert(VN == Lay::VN, "one lane's nodes are one lane's bytes of a block");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long t = *t_dev;
    const RankTab rt = rank_tables<true>(smem_raw, a.B, a.C, t);
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int tiles = (int)(g.Npad / Lay::TN);

    const int n = rt.n;
    if (a.bal_nw > 0) {
        // balanced ranges: this warp's span of (tile, rank) is the tail of one tile, whole tiles, and the head
        // of one more -- the pieces that reach their tile's oldest point (Horner form), then at most one that
        // ends before it
        const long long wp = f16_bal_wp(tiles, n, a.bal_nw);
        const long long lo = (long long)gwarp * wp, hi = min((long long)tiles * n, lo + wp);
        long long tt = lo / n;
        for (; (tt + 1) * n <= hi; ++tt) {
            const long long base = tt * n;
            f16_piece<D, VN, true>(a, rt.e, n, g, (int)tt, (int)max(0ll, lo - base), n, (int)(gwarp - base / wp));
        }
        if (tt * n < hi) {
            const long long base = tt * n;
            f16_piece<D, VN, false>(a, rt.e, n, g, (int)tt, (int)max(0ll, lo - base), (int)(hi - base),
                                    (int)(gwarp - base / wp));
        }
    } else {
        // chunk tasks: tiles x S tasks, chunk-major, warps striding over them -- the chunks before the one that
        // holds the oldest point (running product), then that one (Horner form); chunks past it are empty and
        // the commit does not read them
        const int len = (n + a.S - 1) / a.S;
        const int S_eff = (n + len - 1) / len;
        int task = gwarp;
        for (; task < tiles * (S_eff - 1); task += nwarps) {
            const int chunk = task / tiles;
            f16_piece<D, VN, false>(a, rt.e, n, g, task % tiles, chunk * len, (chunk + 1) * len, chunk);
        }
        for (; task < tiles * S_eff; task += nwarps)
            f16_piece<D, VN, true>(a, rt.e, n, g, task % tiles, (S_eff - 1) * len, n, S_eff - 1);
    }
}

// Byte address of byte b (0..63) of node n's lane in the block of slot l.
template <int D>
__device__ __forceinline__ unsigned char* f16_byte(const CommitF16& a, long long n, long long l, int b) {
    using Lay = F16Layout<D>;
    const long long tile = n / Lay::TN;
    const int q = (int)((n % Lay::TN) / Lay::VN);
    return a.blk + (tile * a.B * a.C + l) * Lay::kBlock + Lay::lane_byte(q, b);
}

// Decode / encode the M values of one vector of node n (M = d*d for Y, NS for Dm) in the block of slot l.
template <int D, bool IS_Y>
__device__ __forceinline__ void f16_get(const CommitF16& a, long long n, long long l, float* v) {
    using Lay = F16Layout<D>;
    constexpr int M = IS_Y ? Lay::DD : Lay::NS;
    const int j = (int)(n % Lay::VN);
    unsigned short u[M];
#pragma unroll
    for (int c = 0; c < M; ++c)
        u[c] = *reinterpret_cast<const unsigned short*>(f16_byte<D>(a, n, l, 2 * (IS_Y ? Lay::y_half(c, j) : Lay::d_half(c, j))));
    const unsigned char eb = *f16_byte<D>(a, n, l, IS_Y ? Lay::ye_byte(j) : Lay::de_byte(j));
    s16_decode<M>(u, eb, v);
}

template <int D, bool IS_Y>
__device__ __forceinline__ void f16_put(const CommitF16& a, long long n, long long l, const float* v) {
    using Lay = F16Layout<D>;
    constexpr int M = IS_Y ? Lay::DD : Lay::NS;
    const int j = (int)(n % Lay::VN);
    unsigned short u[M];
    unsigned char eb;
    s16_encode<M>(v, u, &eb);
#pragma unroll
    for (int c = 0; c < M; ++c)
        *reinterpret_cast<unsigned short*>(f16_byte<D>(a, n, l, 2 * (IS_Y ? Lay::y_half(c, j) : Lay::d_half(c, j)))) = u[c];
    *f16_byte<D>(a, n, l, IS_Y ? Lay::ye_byte(j) : Lay::de_byte(j)) = eb;
}

template <int D, typename N, typename K>
__device__ __forceinline__ void hist_commit_any(Arith<N>, const CommitF16& a, const BlockStep* s_bs, long long Np,
                                                int n, const double* /*kprev*/, const K* ktd, const Chan& p,
                                                N* sig, long long /*t*/) {
    constexpr int DD = D * D;
    constexpr int NS = D == 2 ? 3 : 6;
    float Yn[DD], dn[NS];
    factor_dev<D, float>(ktd, Yn);
    {
        K dd[NS];
        rate_of_strain<D>(ktd, dd);
#pragma unroll
        for (int i = 0; i < NS; ++i) dn[i] = (float)dd[i];
    }
    // the new point as stored (encoded once): its own contribution from the stored, rounded rate
    const long long dst_new = (long long)(a.B - 1) * a.C + s_bs[a.B - 1].head_new;
    N dstored[NS];
    {
        unsigned short um[NS];
        unsigned char ue;
        float f[NS];
        s16_encode<NS>(dn, um, &ue);
        s16_decode<NS>(um, ue, f);
#pragma unroll
        for (int i = 0; i < NS; ++i) dstored[i] = (N)f[i];
    }
    // the chunk records the sweep wrote for this node's tile, the last one the tile's oldest piece (its product
    // not written): balanced ranges cut the tile into pieces; chunk tasks leave the chunks past the oldest
    // point empty
    int npts = 0;
    for (int bb = 0; bb < a.B; ++bb) npts += s_bs[bb].count_prev;
    int S;
    if (a.bal_nw > 0) {
        const long long tiles = Np / F16Layout<D>::TN;
        S = f16_bal_pieces(n / F16Layout<D>::TN, npts, f16_bal_wp(tiles, npts, a.bal_nw));
    } else {
        const int len = (npts + a.S - 1) / a.S;
        S = (npts + len - 1) / len;
    }
    formf_sigma<D, float, float, N>(a.part, S, Np, n, dstored, chan_val<N>(p.G_inf, p.G_inf_f), sig);
    for (int bb = 1; bb < a.B; ++bb) {
        const BlockStep& b = s_bs[bb];
        if (!b.evict) continue;
        int o1 = b.head_prev - (a.C - 1); if (o1 < 0) o1 += a.C;
        int o2 = b.head_prev - (a.C - 2); if (o2 < 0) o2 += a.C;
        const long long s1 = (long long)bb * a.C + o1, s2 = (long long)bb * a.C + o2;
        const long long dst = (long long)(bb - 1) * a.C + s_bs[bb - 1].head_new;
        float Y1[DD], Y2[DD], d1[NS], d2[NS];
        f16_get<D, true>(a, n, s1, Y1);
        f16_get<D, true>(a, n, s2, Y2);
        f16_get<D, false>(a, n, s1, d1);
        f16_get<D, false>(a, n, s2, d2);
        dev_product<D>(Y2, Y1);
#pragma unroll
        for (int c = 0; c < NS; ++c) d1[c] = 0.5f * (d1[c] + d2[c]);
        f16_put<D, true>(a, n, dst, Y2);
        f16_put<D, false>(a, n, dst, d1);
    }
    f16_put<D, true>(a, n, dst_new, Yn);
    f16_put<D, false>(a, n, dst_new, dn);
}

}  // namespace lbk
