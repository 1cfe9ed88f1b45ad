// Matrix-free extended Hubbard ring (Sec. IV.B of arXiv:0802.0748):
//   H = -t sum_{<ij>,s} (c+_is c_js + h.c.) + U sum_i n_i,up n_i,dn + V sum_<ij> n_i n_j
// in the sector with n_up up and n_dn down electrons on L sites.
//
// Basis: index = rank_up * D_dn + rank_dn; rank = position of the occupation
// bit string among all L-bit strings with the same popcount, ascending, which
// is the combinatorial number system sum_j C(pos_j, j + 1) over the set bits
// pos_0 < pos_1 < ...  A hop moves one electron along a bond; with modes
// ordered all up sites then all down sites (Jordan-Wigner) its sign is
// (-1)^(number of same-spin electrons strictly between the two sites).
// Per spin the device builds, for every rank, the list of (target rank, sign)
// of all hops; the diagonal comes from popcounts of the two bit strings.
//
// Apply: a unit is 32 consecutive down-ranks (a "tile") of one up-rank, and
// units are ordered tile-major and visited by all CTAs together, so the up-hop
// gathers x[u'][tile] of concurrently running warps hit the same few column
// tiles of x (L2 reuse); down-hop gathers stay inside the row x[u][:].
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "api_internal.h"
#include "solver_kernel.cuh"
#include "vector_ops.cuh"
#include "hubbard_basis.cuh"

#ifndef SCOCG_RING_TWO_PASS
#define SCOCG_RING_TWO_PASS 0
#endif
#ifndef SCOCG_HOP_GROUP
#define SCOCG_HOP_GROUP 4
#endif

namespace scocg {

template <typename VV> struct Scal;
template <> struct Scal<float2> { using T = float; };
template <> struct Scal<double2> { using T = double; };

// One thread per rank of one spin species.
__global__ void k_hubbard_tables(int L, int k, int D, int ring, uint32_t* states, int32_t* target, int8_t* sign,
                                 int32_t* packed) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const int S = 2 * L;
    const uint32_t s = unrank(r, k, L);
    states[r] = s;
    int cnt = 0;
    const int nb = ring ? L : L - 1;
    for (int b = 0; b < nb; ++b) {
        const int i = b, j = (b + 1) % L;
        for (int dir = 0; dir < 2; ++dir) {
            const int src = dir ? j : i, dst = dir ? i : j;
            if (!((s >> src) & 1u) || ((s >> dst) & 1u)) continue;
            const uint32_t s2 = (s & ~(1u << src)) | (1u << dst);
            const int lo = min(src, dst), hi = max(src, dst);
            const uint32_t between = hi - lo > 1 ? (s & (((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u))) : 0u;
            const int sg = (__popc(between) & 1) ? -1 : 1;
            const int t = (int)rank_of(s2);
            target[(size_t)r * S + cnt] = t;
            sign[(size_t)r * S + cnt] = (int8_t)sg;
            packed[(size_t)r * S + cnt] = (t << 1) | (sg < 0 ? 1 : 0);
            ++cnt;
        }
    }
    for (int c = cnt; c < S; ++c) {
        target[(size_t)r * S + c] = -1;
        sign[(size_t)r * S + c] = 0;
        packed[(size_t)r * S + c] = -1;
    }
}

template <typename R>
struct ApplyHubbard {
    static constexpr int kRowsPerUnit = 32;
    static constexpr int kMap = kMapStrided;
    const uint32_t* st_up;
    const uint32_t* st_dn;
    const int32_t* hop_up;     // packed, [D_up][S]
    const int32_t* hop_dn;     // packed, [D_dn][S]
    int S, D_up, D_dn, L, ring;
    double t, U, V;
    const float2* diagf;     // U cu + V cv as float pairs, index cu * (4 L + 1) + cv
    float t_hi, t_lo;        // t as a float pair
    int64_t n;
    unsigned long long* dbg;

    __device__ __forceinline__ uint32_t partner(uint32_t x) const {
        // bit i of the result = occupation of the bond partner i + 1 (and 0 for i = L - 1 on a ring)
        return (x >> 1) | (ring ? ((x & 1u) << (L - 1)) : 0u);
    }

    // Compensated vectors: the signed hop terms are summed first (each a
    // TwoSum of +-x into a compensated pair, real and imaginary parts packed),
    // then multiplied once by t; the diagonal U n_up n_dn + V n_i n_j and t are
    // taken as float pairs (exact for values such as t = 1, U = 4, V = 1).  The
    // hop lists are read kHopGroup entries at a time: the table entries, then
    // their gathers, are issued together (each list ends at its first -1).
    static constexpr int kHopGroup = SCOCG_HOP_GROUP;
    __device__ __forceinline__ static void hop_acc_df(const int32_t* tab, int S, const float4* base, int64_t stride,
                                                      int64_t lim, unsigned long long* dbg, float2& h, float2& l) {
        for (int j0 = 0; j0 < S; j0 += kHopGroup) {
            int e[kHopGroup];
#pragma unroll
            for (int q = 0; q < kHopGroup; ++q) {
                e[q] = j0 + q < S ? tab[j0 + q] : -1;
                if (e[q] >= 0 && !chk(dbg, 20, e[q] >> 1, lim)) e[q] = -1;
            }
            float4 xv[kHopGroup];
#pragma unroll
            for (int q = 0; q < kHopGroup; ++q) xv[q] = base[(int64_t)(max(e[q], 0) >> 1) * stride];   // entry 0 when ended
#pragma unroll
            for (int q = 0; q < kHopGroup; ++q) {
                if (e[q] >= 0) {
                    const unsigned sg = (unsigned)(e[q] & 1) << 31;    // the sign on the sign bits
                    const float2 xh = make_float2(__uint_as_float(__float_as_uint(xv[q].x) ^ sg),
                                                  __uint_as_float(__float_as_uint(xv[q].y) ^ sg));
                    const float2 xl = make_float2(__uint_as_float(__float_as_uint(xv[q].z) ^ sg),
                                                  __uint_as_float(__float_as_uint(xv[q].w) ^ sg));
                    float2 t, er;
                    pk_two_sum(h, xh, t, er);
                    h = t;
                    l = pk_add(l, pk_add(er, xl));
                }
            }
            if (e[kHopGroup - 1] < 0) break;
        }
    }

    __device__ __forceinline__ bool operator()(int64_t unit, int lane, float4 zs, const float4* x, int64_t& row,
                                               float4& w) const {
        const int u = (int)(unit % D_up);
        const int d = (int)(unit / D_up) * 32 + lane;
        if (d >= D_dn) return false;
        row = (int64_t)u * D_dn + d;
        const uint32_t su = st_up[u], sd = st_dn[d];
        const uint32_t pu = partner(su), pd = partner(sd);
        const int cu = __popc(su & sd);
        const int cv = __popc(su & pu) + __popc(sd & pd) + __popc(su & pd) + __popc(sd & pu);
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        hop_acc_df(hop_dn + (size_t)d * S, S, x + (size_t)u * D_dn, 1, D_dn, dbg, h, l);
        hop_acc_df(hop_up + (size_t)u * S, S, x + d, D_dn, D_up, dbg, h, l);
        pk_norm(h, l);
        const float2 dg = diagf[cu * (4 * L + 1) + cv];
        const dfs zr = df_add(cre(zs), dfs{-dg.x, -dg.y});
        const float4 acc = vcfma(cpack(zr, cim(zs)), x[row], vzero<float4>());   // (z_s - diag) x_row
        float2 ah = hi2(acc), al = lo2(acc);
        // - H's hopping part: + t sum sign x
        pk_acc_prod(ah, al, make_float2(t_hi, t_hi), make_float2(t_lo, t_lo), h, l);
        pk_norm(ah, al);
        w = pk4(ah, al);
        return true;
    }

    // ---- two-pass form (phase A runs pass 1 over all units, a grid barrier,
    // then pass 2; off for the ring, where one pass measured faster: 622 vs
    // 686 us per iteration at 14 sites, while the two-orbital model gains).  Pass 1 visits units row-major
    // (unit = u * tiles + tile: the CTAs share the rows x[u][:] of the down
    // hops) and stores q = (z_s - diag) x + t (down-hop sum) + beta q_old;
    // pass 2 visits them tile-major (unit = tile * D_up + u: the CTAs share the
    // column tiles x[:][tile] of the up hops) and adds t (up-hop sum).
    static constexpr bool kTwoPass = SCOCG_RING_TWO_PASS;
    // the row whose term (unit, lane) adds to the r^T q partial of phase A
    // (the tile-major order of the one-pass apply and of pass 2)
    __device__ __forceinline__ bool row_of(int64_t unit, int lane, int64_t& row) const {
        const int u = (int)(unit % D_up), d = (int)(unit / D_up) * 32 + lane;
        row = (int64_t)u * D_dn + d;
        return d < D_dn;
    }
    __device__ __forceinline__ bool rc_rows(int64_t unit, int lane, int& u, int& d) const {
        const int tiles = (D_dn + 31) / 32;
        u = (int)(unit / tiles);
        d = (int)(unit % tiles) * 32 + lane;
        return d < D_dn;
    }
    __device__ __forceinline__ bool rc_tiles(int64_t unit, int lane, int& u, int& d) const {
        u = (int)(unit % D_up);
        d = (int)(unit / D_up) * 32 + lane;
        return d < D_dn;
    }
    __device__ __forceinline__ int diag_index(int u, int d) const {
        const uint32_t su = st_up[u], sd = st_dn[d];
        const uint32_t pu = partner(su), pd = partner(sd);
        const int cu = __popc(su & sd);
        const int cv = __popc(su & pu) + __popc(sd & pd) + __popc(su & pd) + __popc(sd & pu);
        return cu * (4 * L + 1) + cv;
    }
    __device__ __forceinline__ double diag_of(int u, int d) const {
        const uint32_t su = st_up[u], sd = st_dn[d];
        const uint32_t pu = partner(su), pd = partner(sd);
        const int cu = __popc(su & sd);
        const int cv = __popc(su & pu) + __popc(sd & pd) + __popc(su & pd) + __popc(sd & pu);
        return U * (double)cu + V * (double)cv;
    }

    __device__ __forceinline__ void pass1(int64_t unit, int lane, float4 zs, float4 bp, const float4* x,
                                          float4* q) const {
        int u, d;
        if (!rc_rows(unit, lane, u, d)) return;
        const int64_t row = (int64_t)u * D_dn + d;
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        hop_acc_df(hop_dn + (size_t)d * S, S, x + (size_t)u * D_dn, 1, D_dn, dbg, h, l);
        pk_norm(h, l);
        const float2 dg = diagf[diag_index(u, d)];
        const dfs zr = df_add(cre(zs), dfs{-dg.x, -dg.y});
        const float4 acc = vcfma(cpack(zr, cim(zs)), x[row], vzero<float4>());
        float2 ah = hi2(acc), al = lo2(acc);
        pk_acc_prod(ah, al, make_float2(t_hi, t_hi), make_float2(t_lo, t_lo), h, l);
        pk_norm(ah, al);
        q[row] = vcfma(bp, q[row], pk4(ah, al));
    }
    __device__ __forceinline__ bool pass2(int64_t unit, int lane, const float4* x, float4* q, int64_t& row,
                                          float4& qn) const {
        int u, d;
        if (!rc_tiles(unit, lane, u, d)) return false;
        row = (int64_t)u * D_dn + d;
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        hop_acc_df(hop_up + (size_t)u * S, S, x + d, D_dn, D_up, dbg, h, l);
        pk_norm(h, l);
        const float4 q1 = q[row];
        float2 ah = hi2(q1), al = lo2(q1);
        pk_acc_prod(ah, al, make_float2(t_hi, t_hi), make_float2(t_lo, t_lo), h, l);
        pk_norm(ah, al);
        qn = pk4(ah, al);
        q[row] = qn;
        return true;
    }
    // FP64 and complex64 vectors
    template <typename VV>
    __device__ __forceinline__ VV hop_sum_v(const int32_t* tab, const VV* base, int64_t stride, int64_t lim) const {
        using T = typename Scal<VV>::T;
        VV acc;
        acc.x = 0; acc.y = 0;
        for (int j = 0; j < S; ++j) {
            const int e = tab[j];
            if (e < 0) break;
            if (!chk(dbg, 20, e >> 1, lim)) continue;
            const VV xv = base[(int64_t)(e >> 1) * stride];
            const T c = (e & 1) ? -(T)t : (T)t;
            acc.x += c * xv.x; acc.y += c * xv.y;
        }
        return acc;
    }
    template <typename VV>
    __device__ __forceinline__ void pass1(int64_t unit, int lane, VV zs, VV bp, const VV* x, VV* q) const {
        using T = typename Scal<VV>::T;
        int u, d;
        if (!rc_rows(unit, lane, u, d)) return;
        const int64_t row = (int64_t)u * D_dn + d;
        const VV hs = hop_sum_v(hop_dn + (size_t)d * S, x + (size_t)u * D_dn, 1, D_dn);
        const T zr = zs.x - (T)diag_of(u, d);
        const VV xr = x[row];
        VV w;
        w.x = zr * xr.x - zs.y * xr.y + hs.x;
        w.y = zr * xr.y + zs.y * xr.x + hs.y;
        q[row] = vcfma(bp, q[row], w);
    }
    template <typename VV>
    __device__ __forceinline__ bool pass2(int64_t unit, int lane, const VV* x, VV* q, int64_t& row, VV& qn) const {
        int u, d;
        if (!rc_tiles(unit, lane, u, d)) return false;
        row = (int64_t)u * D_dn + d;
        const VV hs = hop_sum_v(hop_up + (size_t)u * S, x + d, D_dn, D_up);
        qn = q[row];
        qn.x += hs.x; qn.y += hs.y;
        q[row] = qn;
        return true;
    }

    template <typename VV>
    __device__ __forceinline__ bool operator()(int64_t unit, int lane, VV zs, const VV* x, int64_t& row,
                                               VV& w) const {
        using T = typename Scal<VV>::T;
        const int u = (int)(unit % D_up);
        const int d = (int)(unit / D_up) * 32 + lane;
        if (d >= D_dn) return false;
        row = (int64_t)u * D_dn + d;
        const uint32_t su = st_up[u], sd = st_dn[d];
        const uint32_t pu = partner(su), pd = partner(sd);
        const int cu = __popc(su & sd);
        const int cv = __popc(su & pu) + __popc(sd & pd) + __popc(su & pd) + __popc(sd & pu);
        const T diag = (T)U * (T)cu + (T)V * (T)cv;
        VV acc;
        {
            const VV xr = x[row];
            const T zr = zs.x - diag;
            acc.x = zr * xr.x - zs.y * xr.y;
            acc.y = zr * xr.y + zs.y * xr.x;
        }
        const T tt = (T)t;
        const VV* xrow = x + (size_t)u * D_dn;
        for (int j = 0; j < S; ++j) {
            const int e = hop_dn[(size_t)d * S + j];
            if (e < 0) break;
            if (!chk(dbg, 20, e >> 1, D_dn)) continue;
            const VV xv = xrow[e >> 1];
            const T c = (e & 1) ? -tt : tt;
            acc.x += c * xv.x; acc.y += c * xv.y;
        }
        for (int j = 0; j < S; ++j) {
            const int e = hop_up[(size_t)u * S + j];
            if (e < 0) break;
            if (!chk(dbg, 21, e >> 1, D_up)) continue;
            const VV xv = x[(size_t)(e >> 1) * D_dn + d];
            const T c = (e & 1) ? -tt : tt;
            acc.x += c * xv.x; acc.y += c * xv.y;
        }
        w = acc;
        return true;
    }
};

template <typename R>
static ApplyHubbard<R> make_apply(const Hubbard& hb) {
    ApplyHubbard<R> ap;
    ap.st_up = hb.d_states;
    ap.st_dn = hb.d_states + hb.Dmax;
    ap.S = 2 * hb.L;
    ap.hop_up = hb.d_hop_packed;
    ap.hop_dn = hb.d_hop_packed + (size_t)hb.Dmax * ap.S;
    ap.D_up = hb.D_up; ap.D_dn = hb.D_dn; ap.L = hb.L;
    ap.ring = hb.periodic && hb.L >= 3;
    ap.t = hb.t; ap.U = hb.U; ap.V = hb.V;
    ap.diagf = hb.d_diagf;
    ap.t_hi = (float)hb.t;
    ap.t_lo = (float)(hb.t - (double)ap.t_hi);
    ap.n = (int64_t)hb.D_up * hb.D_dn;
    ap.dbg = nullptr;
    return ap;
}

int hubbard_max_ctas(const Hubbard& hb, int prec, int num_sms, size_t dyn_smem) {
    if (hb.model == 1) return hubbard2_max_ctas(hb, prec, num_sms, dyn_smem);
    int nb = 0;
    cudaError_t e =
        prec == SCOCG_MIXED
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<float, ApplyHubbard<float>>, kBlock,
                                                            dyn_smem)
        : prec == SCOCG_MIXED_DF
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<DF, ApplyHubbard<float>>, kBlock,
                                                            dyn_smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<double, ApplyHubbard<double>>,
                                                            kBlock, dyn_smem);
    (void)hb;
    return e == cudaSuccess ? nb * num_sms : 0;
}

template <typename R>
cudaError_t hubbard_launch_solve(const SolveArgs<R>& a, const Hubbard& hb, int grid, cudaStream_t st) {
    if (hb.model == 1) return hubbard2_launch_solve<R>(a, hb, grid, st);
    using W = typename ValT<R>::T;
    ApplyHubbard<W> ap = make_apply<W>(hb);
    ap.dbg = a.dbg;
    void* args[] = {(void*)&a, (void*)&ap};
    const size_t smem = a.Xf ? (size_t)a.K * kFullSmem : 0;
    // a continuation of a stopped solve runs its own instantiation
    const void* kern = a.resume ? (const void*)cocg_persistent<R, ApplyHubbard<W>, true>
                                : (const void*)cocg_persistent<R, ApplyHubbard<W>, false>;
    if (smem > 0)   // above the 48 KB default together with the static part
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kBlock), args, smem, st);
}
template cudaError_t hubbard_launch_solve<double>(const SolveArgs<double>&, const Hubbard&, int, cudaStream_t);
template cudaError_t hubbard_launch_solve<float>(const SolveArgs<float>&, const Hubbard&, int, cudaStream_t);
template cudaError_t hubbard_launch_solve<DF>(const SolveArgs<DF>&, const Hubbard&, int, cudaStream_t);

template <typename VV, class Apply>
__global__ void __launch_bounds__(256) k_hub_apply(Apply ap, int64_t nunits, VV zs, const VV* x, VV* y) {
    const int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (u >= nunits) return;
    int64_t row;
    VV w;
    if (ap(u, threadIdx.x & 31, zs, x, row, w)) y[row] = w;
}

cudaError_t hubbard_apply(const Hubbard& hb, int prec, double2 z, const void* x, void* y, cudaStream_t st) {
    if (hb.model == 1) return hubbard2_apply(hb, prec, z, x, y, st);
    const unsigned blocks = (unsigned)((hb.nunits * 32 + 255) / 256);
    if (prec == SCOCG_MIXED)
        k_hub_apply<float2><<<blocks, 256, 0, st>>>(make_apply<float>(hb), hb.nunits,
                                                    make_float2((float)z.x, (float)z.y), (const float2*)x, (float2*)y);
    else if (prec == SCOCG_MIXED_DF)
        k_hub_apply<float4><<<blocks, 256, 0, st>>>(make_apply<float>(hb), hb.nunits, df_from(z), (const float4*)x,
                                                    (float4*)y);
    else
        k_hub_apply<double2><<<blocks, 256, 0, st>>>(make_apply<double>(hb), hb.nunits, z, (const double2*)x,
                                                     (double2*)y);
    return cudaGetLastError();
}

constexpr int kHopBatch = 4;
constexpr int kMaxSites = 16;   // scocg_create_hubbard accepts L <= 16

// acc + sum over the hop list tab[0..S) (ended by -1) of sign * base[target * stride],
// sign = -1 where bit 0 of the entry is set, added in list order
__device__ __forceinline__ double hop_sum(const int32_t* tab, int S, const double* base, int64_t stride, double acc) {
    for (int j0 = 0; j0 < S; j0 += kHopBatch) {
        int e[kHopBatch];
        double xv[kHopBatch];
#pragma unroll
        for (int q = 0; q < kHopBatch; ++q) e[q] = j0 + q < S ? tab[j0 + q] : -1;
#pragma unroll
        for (int q = 0; q < kHopBatch; ++q)
            if (e[q] >= 0) xv[q] = base[(int64_t)(e[q] >> 1) * stride];
#pragma unroll
        for (int q = 0; q < kHopBatch; ++q) {
            if (e[q] < 0) return acc;
            acc += __longlong_as_double(__double_as_longlong(xv[q]) ^ ((long long)(e[q] & 1) << 63));
        }
    }
    return acc;
}

// Real FP64 operator of the ground-state iteration: y = (H - sigma) x - beta x_prev
// (x_prev and beta optional), same unit order as the solver's apply, and the
// block's partial of x^T y in part[blockIdx.x].  A launch whose *skip is set
// does nothing.
__global__ void __launch_bounds__(kVecBlock) k_hub_hx(ApplyHubbard<double> ap, int64_t nunits, const double* x,
                                                      double* y, const double* xprev, const double* beta,
                                                      double sigma, const int* skip, double* part) {
    if (skip && *skip) return;
    // diagonal minus sigma for every (double occupancies, neighbour pairs):
    // U cu + V cv - sigma, cu <= L, cv <= 4 L, built once per block
    __shared__ double s_diag[(kMaxSites + 1) * (4 * kMaxSites + 1)];
    const int ncv = 4 * ap.L + 1;
    for (int i = threadIdx.x; i < (ap.L + 1) * ncv; i += kVecBlock)
        s_diag[i] = fma(ap.U, (double)(i / ncv), fma(ap.V, (double)(i % ncv), -sigma));
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)kVecBlock + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kVecBlock) >> 5;
    const double bp = (xprev && beta) ? *beta : 0.0;
    double acc = 0.0;
    for (int64_t unit = w0; unit < nunits; unit += nw) {
        const int u = (int)(unit % ap.D_up);
        const int d = (int)(unit / ap.D_up) * 32 + lane;
        if (d >= ap.D_dn) continue;
        const int64_t row = (int64_t)u * ap.D_dn + d;
        const uint32_t su = ap.st_up[u], sd = ap.st_dn[d];
        const uint32_t pu = ap.partner(su), pd = ap.partner(sd);
        const int cu = __popc(su & sd);
        const int cv = __popc(su & pu) + __popc(sd & pd) + __popc(su & pd) + __popc(sd & pu);
        const double xi = x[row];
        double hop = 0.0;   // sum of sign * x over the hops; H's hopping part is -t times it
        // hops in batches of kHopBatch: the table entries, then the gathers, are
        // issued together; the list of a string ends at its first -1, and the
        // sign is put on the gathered value's sign bit (one FP64 add per hop)
        const double* xrow = x + (size_t)u * ap.D_dn;
        hop = hop_sum(ap.hop_dn + (size_t)d * ap.S, ap.S, xrow, 1, hop);
        hop = hop_sum(ap.hop_up + (size_t)u * ap.S, ap.S, x + d, ap.D_dn, hop);
        double yi = fma(s_diag[cu * ncv + cv], xi, -ap.t * hop);
        if (xprev) yi = fma(-bp, xprev[row], yi);
        y[row] = yi;
        acc = fma(xi, yi, acc);
    }
    block_partial(acc, part);
}

cudaError_t hubbard_hx(const Hubbard& hb, const double* x, double* y, const double* xprev, const double* beta,
                       double sigma, const int* skip, double* part, int grid, cudaStream_t st) {
    if (hb.model == 1) return hubbard2_hx(hb, x, y, xprev, beta, sigma, skip, part, grid, st);
    k_hub_hx<<<grid, kVecBlock, 0, st>>>(make_apply<double>(hb), hb.nunits, x, y, xprev, beta, sigma, skip, part);
    return cudaGetLastError();
}

// c_{site,spin} or c+_{site,spin} from the sector of `src` into the sector of
// this handle: one thread per target basis state.  The source state is the
// target with mode (site, spin) flipped back; with modes ordered all up sites
// then all down sites, the Jordan-Wigner sign is (-1)^(occupied modes before
// the flipped one) in the source state.  Output complex128 with zero imaginary
// part (a right-hand side of the shifted solve).
__global__ void k_excite(int site, int spin, int create, int n_up_src, int D_dn_src, const uint32_t* st_up_t,
                         const uint32_t* st_dn_t, int D_up_t, int D_dn_t, const double* psi, double2* out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)D_up_t * D_dn_t) return;
    const int ut = (int)(t / D_dn_t), dt = (int)(t % D_dn_t);
    uint32_t su = st_up_t[ut], sd = st_dn_t[dt];
    const uint32_t bit = 1u << site;
    const uint32_t s_t = spin ? sd : su;
    double v = 0.0;
    if (((s_t & bit) != 0u) == (create != 0)) {
        if (spin) sd ^= bit; else su ^= bit;
        const uint32_t s_src = spin ? sd : su;
        const int before = __popc(s_src & (bit - 1u)) + (spin ? n_up_src : 0);
        const int64_t src = spin ? (int64_t)ut * D_dn_src + rank_of(sd) : rank_of(su) * D_dn_src + dt;
        const double p = psi[src];
        v = (before & 1) ? -p : p;
    }
    out[t] = make_double2(v, 0.0);
}

}  // namespace scocg

using namespace scocg;

extern "C" int scocg_create_hubbard(scocg_handle* out, int L, int n_up, int n_dn, double t, double U, double V,
                                    int periodic, const scocg_opts* opts, void* cuda_stream) {
    if (!out) return SCOCG_ERR_INVALID;
    *out = nullptr;
    if (L < 2 || L > 16 || n_up < 0 || n_dn < 0 || n_up > L || n_dn > L || !std::isfinite(t) ||
        !std::isfinite(U) || !std::isfinite(V))
        return SCOCG_ERR_INVALID;
    scocg_ctx* h = new (std::nothrow) scocg_ctx();
    if (!h) return SCOCG_ERR_OOM;
    int st = init_ctx(h, opts, cuda_stream);
    if (st != SCOCG_OK) { h->free_all(); delete h; return st; }
    Hubbard& hb = h->hub;
    hb.L = L; hb.n_up = n_up; hb.n_dn = n_dn; hb.periodic = periodic ? 1 : 0;
    hb.t = t; hb.U = U; hb.V = V;
    hb.D_up = (int)binom(L, n_up);
    hb.D_dn = (int)binom(L, n_dn);
    hb.Dmax = std::max(hb.D_up, hb.D_dn);
    const int S = 2 * L;
    hb.nunits = (int64_t)hb.D_up * ((hb.D_dn + 31) / 32);
    h->kind = HandleKind::kHubbard;
    h->n = (int64_t)hb.D_up * hb.D_dn;
    h->nnz = 0;
    const size_t tab = (size_t)hb.Dmax * S;
    cudaError_t e = cudaMalloc(&hb.d_states, sizeof(uint32_t) * 2 * hb.Dmax);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_hop_target, sizeof(int32_t) * 2 * tab);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_hop_sign, sizeof(int8_t) * 2 * tab);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_hop_packed, sizeof(int32_t) * 2 * tab);
    const int ring = (periodic && L >= 3) ? 1 : 0;
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
        const int D = sp ? hb.D_dn : hb.D_up, k = sp ? n_dn : n_up;
        k_hubbard_tables<<<(D + 127) / 128, 128, 0, h->stream>>>(L, k, D, ring, hb.d_states + (size_t)sp * hb.Dmax,
                                                                 hb.d_hop_target + sp * tab, hb.d_hop_sign + sp * tab,
                                                                 hb.d_hop_packed + sp * tab);
        e = cudaGetLastError();
    }
    {   // the diagonal U cu + V cv for every count pair, as float pairs
        const int ncv = 4 * L + 1;
        std::vector<float2> dg((size_t)(L + 1) * ncv);
        for (int cu = 0; cu <= L; ++cu)
            for (int cv = 0; cv < ncv; ++cv) {
                const double v = U * (double)cu + V * (double)cv;
                const float hi = (float)v;
                dg[(size_t)cu * ncv + cv] = make_float2(hi, (float)(v - (double)hi));
            }
        if (e == cudaSuccess) e = cudaMalloc(&hb.d_diagf, sizeof(float2) * dg.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hb.d_diagf, dg.data(), sizeof(float2) * dg.size(), cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    hb.table_bytes = (double)(hb.D_up + hb.D_dn) * (4.0 + 4.0 * S);
    if (e != cudaSuccess) { st = cuda_status(e); h->free_all(); delete h; return st; }
    *out = h;
    return SCOCG_OK;
}

extern "C" int scocg_hubbard_tables(scocg_handle h, int spin, int32_t* dim, uint32_t* states, int32_t* hop_target,
                                    int8_t* hop_sign) {
    if (!h || h->kind != HandleKind::kHubbard || (spin != 0 && spin != 1) || !dim) return SCOCG_ERR_INVALID;
    const Hubbard& hb = h->hub;
    const int D = spin ? hb.D_dn : hb.D_up;
    const size_t S = 2 * hb.L, tab = (size_t)hb.Dmax * S;
    *dim = D;
    cudaError_t e = cudaSuccess;
    if (states) e = cudaMemcpy(states, hb.d_states + (size_t)spin * hb.Dmax, sizeof(uint32_t) * D, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hop_target)
        e = cudaMemcpy(hop_target, hb.d_hop_target + spin * tab, sizeof(int32_t) * D * S, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hop_sign)
        e = cudaMemcpy(hop_sign, hb.d_hop_sign + spin * tab, sizeof(int8_t) * D * S, cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

extern "C" int scocg_excite(scocg_handle from, scocg_handle to, int site, int spin, int create, const double* psi,
                            void* out) {
    if (!from || !to || !psi || !out || from->kind != HandleKind::kHubbard || to->kind != HandleKind::kHubbard)
        return SCOCG_ERR_INVALID;
    const Hubbard& a = from->hub;
    const Hubbard& b = to->hub;
    const int d = create ? 1 : -1;
    if (a.L != b.L || site < 0 || site >= a.L || (spin != 0 && spin != 1) || (create != 0 && create != 1))
        return SCOCG_ERR_INVALID;
    const int tu = a.n_up + (spin == 0 ? d : 0), td = a.n_dn + (spin == 1 ? d : 0);
    if (b.n_up != tu || b.n_dn != td) return SCOCG_ERR_INVALID;
    const int64_t n_t = (int64_t)b.D_up * b.D_dn;
    if (n_t == 0) return SCOCG_OK;
    if (from->stream != to->stream) {   // psi may still be written on the source handle's stream
        cudaError_t e = cudaStreamSynchronize(from->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    k_excite<<<(unsigned)((n_t + 255) / 256), 256, 0, to->stream>>>(site, spin, create, a.n_up, a.D_dn,
                                                                     b.d_states, b.d_states + b.Dmax, b.D_up, b.D_dn,
                                                                     psi, (double2*)out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(to->stream);
    return cuda_status(e);
}
