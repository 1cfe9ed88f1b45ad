// Matrix-free two-orbital (doubly degenerate) extended Hubbard model on a
// cluster (Sec. IV.B of arXiv:0802.0748: two orbitals per site, inter-site
// Coulomb V; the paper's sqrt(8) x sqrt(8) problem has 64,128,064 states):
//
//   H = sum_{bonds (i,j)} sum_{a,b} sum_s t^{ij}_{ab} (c+_{ias} c_{jbs} + h.c.)
//     + U sum_{ia} n_{ia up} n_{ia dn} + U' sum_i n_{i0} n_{i1} - J sum_{is} n_{i0s} n_{i1s}
//     + J sum_{is} c+_{i0s} c+_{i1s'} c_{i0s'} c_{i1s}
//     + J' sum_i (c+_{i0 up} c+_{i0 dn} c_{i1 dn} c_{i1 up} + h.c.) + V sum_{bonds} n_i n_j
//
// Modes per spin: 2 i + a (site i, orbital a); all up-spin modes, then all
// down-spin modes (Jordan-Wigner order).  Basis index rank_up * D_dn +
// rank_dn, ranks as in hubbard_basis.cuh.
//
// Per spin the device builds for every rank:
//   * the hop list: (target rank, amplitude index b*4 + a*2 + a', sign) of
//     every c+_{ia} c_{ja'} and c+_{ja'} c_{ia} of every bond b = (i, j);
//   * the orbital-move list: per site, the rank reached by moving its single
//     electron to the other orbital (none when the site holds 0 or 2 of this
//     spin).  The spin-flip and pair-hopping terms are products of one such
//     move of each spin on the same site (the two moves to different orbitals:
//     J; to the same orbital: J'); neighbouring modes, so no Jordan-Wigner sign;
//   * the diagonal terms of that spin alone ((U' - J) n_{i0} n_{i1} and
//     V sum_bonds n_i n_j), and its site occupations n_i and their neighbour
//     sums (A n)_i as nibbles for the cross-spin V term.
// The apply adds, per row (u, d): the cross-spin diagonal U c_U + U' c_U' +
// V c_V from integer counts (tables of small multiples), the down hops inside
// the row x[u][:], the up hops x[u'][d], and the joint moves x[u'][d'].
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "api_internal.h"
#include "hubbard_basis.cuh"
#include "solver_kernel.cuh"
#include "vector_ops.cuh"

namespace scocg {

constexpr int kMaxSites2 = 16;       // 2 ns <= 32 modes per spin
constexpr int kMaxBonds2 = 32;       // amplitude index b*4 + a*2 + a' < 128 (7 bits)
constexpr int kCross2 = 257;         // counts 0..256 of the cross-spin diagonal tables (8 per bond at most)
#ifndef SCOCG_H2_GROUP
#define SCOCG_H2_GROUP 4
#endif
constexpr int kHop2Group = SCOCG_H2_GROUP;   // hop entries read (and gathered) together
#ifndef SCOCG_H2_UMAJOR
#define SCOCG_H2_UMAJOR 0
#endif

__device__ __forceinline__ int parity_sign(int c) { return (c & 1) ? -1 : 1; }

// One thread per rank of one spin species: the basis string, the hop list, the
// orbital-move list and the spin's own diagonal terms.
__global__ void k_hubbard2_tables(int ns, int nb, int k, int D, const int32_t* bonds, double Up, double J, double V,
                                  int S2, uint32_t* states, int32_t* hop, int32_t* orb, uint32_t* nib, double* self,
                                  float2* selff) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= D) return;
    const int M = 2 * ns;
    const uint32_t s = unrank(r, k, M);
    states[r] = s;
    int cnt = 0;
    for (int b = 0; b < nb; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        for (int a = 0; a < 2; ++a)
            for (int a2 = 0; a2 < 2; ++a2) {
                const int amp = b * 4 + a * 2 + a2;
                for (int dir = 0; dir < 2; ++dir) {   // c+_{dst} c_{src}
                    const int dst = dir ? 2 * j + a2 : 2 * i + a, src = dir ? 2 * i + a : 2 * j + a2;
                    if (!((s >> src) & 1u) || ((s >> dst) & 1u)) continue;
                    const uint32_t s1 = s & ~(1u << src);
                    const int sg = parity_sign(__popc(s & ((1u << src) - 1u)) + __popc(s1 & ((1u << dst) - 1u)));
                    const int t = (int)rank_of(s1 | (1u << dst));
                    if (cnt < S2) hop[(size_t)cnt * D + r] = (t << 8) | (amp << 1) | (sg < 0 ? 1 : 0);
                    ++cnt;
                }
            }
    }
    for (int c = cnt; c < S2; ++c) hop[(size_t)c * D + r] = -1;
    uint32_t ni = 0, ani = 0;
    double sv = 0.0;
    int same = 0;
    for (int i = 0; i < ns; ++i) {
        const uint32_t o = (s >> (2 * i)) & 3u;
        int32_t mv = -1;
        if (o == 1u || o == 2u) {   // one electron: move it to the other orbital
            const int dst = o == 1u ? 1 : 0;
            mv = (int32_t)(rank_of(s ^ (3u << (2 * i))) << 1) | dst;
        }
        orb[(size_t)i * D + r] = mv;
        ni |= (uint32_t)__popc(o) << (4 * i);
        same += o == 3u;
    }
    for (int b = 0; b < nb; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        const uint32_t n_i = (ni >> (4 * i)) & 15u, n_j = (ni >> (4 * j)) & 15u;
        sv += (double)(n_i * n_j);
        ani += n_j << (4 * i);
        ani += n_i << (4 * j);
    }
    nib[2 * (size_t)r] = ni;
    nib[2 * (size_t)r + 1] = ani;
    const double d = (Up - J) * (double)same + V * sv;
    self[r] = d;
    const float hi = (float)d;
    selff[r] = make_float2(hi, (float)(d - (double)hi));
}

template <typename R>
struct ApplyHubbard2 {
    static constexpr int kRowsPerUnit = 32;
    static constexpr int kMap = kMapStrided;
    const uint32_t* st_up;
    const uint32_t* st_dn;
    const int32_t* hop_up;
    const int32_t* hop_dn;     // [S2][D] (slot-major: a warp's 32 ranks read one line per slot)
    const int32_t* orb_up;
    const int32_t* orb_dn;     // [ns][D]
    const uint32_t* nib_up;
    const uint32_t* nib_dn;    // [D][2]
    const double* self_up;
    const double* self_dn;
    const float2* selff_up;
    const float2* selff_dn;
    const double* amp;         // [4 nb]
    const float4* ampf;        // [4 nb][2]: the signed amplitude (sign t) as (hi, hi, lo, lo)
    const double* cross;       // [3][kCross2]: U c, U' c, V c
    const float2* crossf;
    int S2, ns, D_up, D_dn;
    double J, Jp;
    float Jh, Jl, Ph, Pl;      // -J and -J' as float pairs (hi, lo)
    int64_t n;
    unsigned long long* dbg;

    // Row (u, d) of (unit, lane).  Units are visited by all CTAs together in
    // unit order; up-major (unit = u * tiles + tile) keeps the rows x[u][:] of
    // the down hops and the joint moves' rows in cache, tile-major (unit =
    // tile * D_up + u) the column tiles x[:][tile] of the up hops.
    __device__ __forceinline__ void unit_rc(int64_t unit, int lane, int& u, int& d) const {
#if SCOCG_H2_UMAJOR
        const int tiles = (D_dn + 31) / 32;
        u = (int)(unit / tiles);
        d = (int)(unit % tiles) * 32 + lane;
#else
        u = (int)(unit % D_up);
        d = (int)(unit / D_up) * 32 + lane;
#endif
    }

    // the cross-spin diagonal counts of row (u, d)
    __device__ __forceinline__ void counts(uint32_t su, uint32_t sd, int u, int d, int& cu, int& cp, int& cv) const {
        const uint32_t ev = 0x55555555u;
        cu = __popc(su & sd);
        cp = __popc(su & (sd >> 1) & ev) + __popc(sd & (su >> 1) & ev);
        const uint32_t nu = nib_up[2 * (size_t)u], and_ = nib_dn[2 * (size_t)d + 1];
        int c = 0;
#pragma unroll 4
        for (int i = 0; i < ns; ++i) c += (int)(((nu >> (4 * i)) & 15u) * ((and_ >> (4 * i)) & 15u));
        cv = c;
    }

    // Compensated vectors: per hop a product of the amplitude (float pair)
    // and x (exact to the pair precision) summed by TwoSum, real and imaginary
    // parts packed; the joint moves are summed by coefficient (J or J') and
    // multiplied once; the diagonal from the spins' own terms and the
    // cross-spin tables, as float pairs.
    __device__ __forceinline__ void hops_df(const int32_t* tab, int64_t tstride, const float4* base, int64_t stride,
                                            int64_t lim, float2& h, float2& l) const {
        for (int j0 = 0; j0 < S2; j0 += kHop2Group) {
            int e[kHop2Group];
#pragma unroll
            for (int q = 0; q < kHop2Group; ++q) {
                e[q] = j0 + q < S2 ? tab[(int64_t)(j0 + q) * tstride] : -1;
                if (e[q] >= 0 && !chk(dbg, 22, e[q] >> 8, lim)) e[q] = -1;
            }
            // every load is issued (an ended list reads entry 0) and only the
            // valid entries are added
            float4 xv[kHop2Group];
#pragma unroll
            for (int q = 0; q < kHop2Group; ++q) xv[q] = base[(int64_t)(max(e[q], 0) >> 8) * stride];
#pragma unroll
            for (int q = 0; q < kHop2Group; ++q) {
                if (e[q] >= 0) {
                    const float4 t = ampf[e[q] & 255];
                    pk_acc_prod(h, l, make_float2(t.x, t.y), make_float2(t.z, t.w), hi2(xv[q]), lo2(xv[q]));
                }
            }
            if (e[kHop2Group - 1] < 0) break;
        }
    }

    // joint moves (spin flip: J, pair hopping: J'), summed separately
    __device__ __forceinline__ void joint_df(int u, int d, const float4* x, float2& hj, float2& lj, float2& hp,
                                             float2& lp) const {
        for (int i = 0; i < ns; ++i) {
            const int32_t mu = orb_up[(size_t)i * D_up + u], md = orb_dn[(size_t)i * D_dn + d];
            if (mu < 0 || md < 0) continue;
            const int tu = mu >> 1, td = md >> 1;
            if (!chk(dbg, 23, tu, D_up) || !chk(dbg, 24, td, D_dn)) continue;
            const float4 xv = x[(size_t)tu * D_dn + td];
            float2 t, er;
            if ((mu & 1) != (md & 1)) {
                pk_two_sum(hj, hi2(xv), t, er);
                hj = t; lj = pk_add(lj, pk_add(er, lo2(xv)));
            } else {
                pk_two_sum(hp, hi2(xv), t, er);
                hp = t; lp = pk_add(lp, pk_add(er, lo2(xv)));
            }
        }
        pk_norm(hj, lj);
        pk_norm(hp, lp);
    }
    // w = (z_s - diag) x_row - (hops h + l) - J (hj + lj) - J' (hp + lp)
    __device__ __forceinline__ float4 combine_df(int u, int d, int cu, int cp, int cv, float4 zs, float4 xr,
                                                 float2 h, float2 l, float2 hj, float2 lj, float2 hp,
                                                 float2 lp) const {
        pk_norm(h, l);
        const float2 d0 = selff_up[u], d1 = selff_dn[d];
        const float2 c0 = crossf[min(cu, kCross2 - 1)], c1 = crossf[kCross2 + min(cp, kCross2 - 1)],
                     c2v = crossf[2 * kCross2 + min(cv, kCross2 - 1)];
        const dfs dg = df_add(df_add(dfs{d0.x, d0.y}, dfs{d1.x, d1.y}),
                              df_add(dfs{c0.x, c0.y}, df_add(dfs{c1.x, c1.y}, dfs{c2v.x, c2v.y})));
        const dfs zr = df_add(cre(zs), df_neg(dg));
        const float4 acc = vcfma(cpack(zr, cim(zs)), xr, vzero<float4>());
        float2 ah = hi2(acc), al = lo2(acc);
        float2 s, e;
        pk_two_sum(ah, pk_neg(h), s, e);
        ah = s;
        al = pk_add(al, pk_sub(e, l));
        pk_acc_prod(ah, al, make_float2(Jh, Jh), make_float2(Jl, Jl), hj, lj);
        pk_acc_prod(ah, al, make_float2(Ph, Ph), make_float2(Pl, Pl), hp, lp);
        pk_norm(ah, al);
        return pk4(ah, al);
    }

    __device__ __forceinline__ bool operator()(int64_t unit, int lane, float4 zs, const float4* x, int64_t& row,
                                               float4& w) const {
        int u, d;
        unit_rc(unit, lane, u, d);
        if (d >= D_dn) return false;
        row = (int64_t)u * D_dn + d;
        const uint32_t su = st_up[u], sd = st_dn[d];
        int cu, cp, cv;
        counts(su, sd, u, d, cu, cp, cv);
        // hops: h + l = (H's hopping part) x = sum t sign x over the hop lists
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        hops_df(hop_dn + d, D_dn, x + (size_t)u * D_dn, 1, D_dn, h, l);
        hops_df(hop_up + u, D_up, x + d, D_dn, D_up, h, l);
        float2 hj = make_float2(0.f, 0.f), lj = hj, hp = hj, lp = hj;
        joint_df(u, d, x, hj, lj, hp, lp);
        w = combine_df(u, d, cu, cp, cv, zs, x[row], h, l, hj, lj, hp, lp);
        return true;
    }

    // ---- two-pass form used by the persistent solve: pass 1 over the units
    // row-major (the CTAs share the rows x[u][:] of the down hops and the few
    // rows of the joint moves) stores q = (z_s - diag) x - (down hops and
    // joint moves) + beta q_old; pass 2 tile-major (the CTAs share the column
    // tiles x[:][tile] of the up hops) subtracts the up hops.
    static constexpr bool kTwoPass = true;
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
    __device__ __forceinline__ float4 pass1_w(int u, int d, float4 zs, const float4* x) const {
        const int64_t row = (int64_t)u * D_dn + d;
        const uint32_t su = st_up[u], sd = st_dn[d];
        int cu, cp, cv;
        counts(su, sd, u, d, cu, cp, cv);
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        hops_df(hop_dn + d, D_dn, x + (size_t)u * D_dn, 1, D_dn, h, l);
        float2 hj = make_float2(0.f, 0.f), lj = hj, hp = hj, lp = hj;
        joint_df(u, d, x, hj, lj, hp, lp);
        return combine_df(u, d, cu, cp, cv, zs, x[row], h, l, hj, lj, hp, lp);
    }
    __device__ __forceinline__ void pass1(int64_t unit, int lane, float4 zs, float4 bp, const float4* x,
                                          float4* q) const {
        int u, d;
        if (!rc_rows(unit, lane, u, d)) return;
        const int64_t row = (int64_t)u * D_dn + d;
        q[row] = vcfma(bp, q[row], pass1_w(u, d, zs, x));
    }
    __device__ __forceinline__ bool pass2(int64_t unit, int lane, const float4* x, float4* q, int64_t& row,
                                          float4& qn) const {
        int u, d;
        if (!rc_tiles(unit, lane, u, d)) return false;
        row = (int64_t)u * D_dn + d;
        float2 h = make_float2(0.f, 0.f), l = make_float2(0.f, 0.f);
        hops_df(hop_up + u, D_up, x + d, D_dn, D_up, h, l);
        pk_norm(h, l);
        const float4 q1 = q[row];
        float2 s, e;
        pk_two_sum(hi2(q1), pk_neg(h), s, e);
        e = pk_add(e, pk_sub(lo2(q1), l));
        pk_norm(s, e);
        qn = pk4(s, e);
        q[row] = qn;
        return true;
    }
    // FP64 (double2) and complex64 (float2) vectors
    template <typename VV>
    __device__ __forceinline__ VV hops_v(const int32_t* tab, int64_t ts, const VV* base, int64_t stride,
                                         int64_t lim) const {
        using T = decltype(base->x);
        VV acc;
        acc.x = 0; acc.y = 0;
        for (int j = 0; j < S2; ++j) {
            const int e = tab[(int64_t)j * ts];
            if (e < 0) break;
            if (!chk(dbg, 22, e >> 8, lim)) continue;
            const VV xv = base[(int64_t)(e >> 8) * stride];
            const T t = (T)amp[(e >> 1) & 127];
            const T c = (e & 1) ? -t : t;   // H's element
            acc.x += c * xv.x; acc.y += c * xv.y;
        }
        return acc;
    }
    template <typename VV>
    __device__ __forceinline__ void pass1(int64_t unit, int lane, VV zs, VV bp, const VV* x, VV* q) const {
        using T = decltype(zs.x);
        int u, d;
        if (!rc_rows(unit, lane, u, d)) return;
        const int64_t row = (int64_t)u * D_dn + d;
        const uint32_t su = st_up[u], sd = st_dn[d];
        int cu, cp, cv;
        counts(su, sd, u, d, cu, cp, cv);
        const T diag = (T)(self_up[u] + self_dn[d] + cross[min(cu, kCross2 - 1)] +
                           cross[kCross2 + min(cp, kCross2 - 1)] + cross[2 * kCross2 + min(cv, kCross2 - 1)]);
        const VV hs = hops_v(hop_dn + d, D_dn, x + (size_t)u * D_dn, 1, D_dn);
        VV acc;
        const VV xr = x[row];
        const T zr = zs.x - diag;
        acc.x = zr * xr.x - zs.y * xr.y - hs.x;
        acc.y = zr * xr.y + zs.y * xr.x - hs.y;
        for (int i = 0; i < ns; ++i) {
            const int32_t mu = orb_up[(size_t)i * D_up + u], md = orb_dn[(size_t)i * D_dn + d];
            if (mu < 0 || md < 0) continue;
            const int tu = mu >> 1, td = md >> 1;
            if (!chk(dbg, 23, tu, D_up) || !chk(dbg, 24, td, D_dn)) continue;
            const VV xv = x[(size_t)tu * D_dn + td];
            const T c = -(T)((mu & 1) != (md & 1) ? J : Jp);
            acc.x += c * xv.x; acc.y += c * xv.y;
        }
        q[row] = vcfma(bp, q[row], acc);
    }
    template <typename VV>
    __device__ __forceinline__ bool pass2(int64_t unit, int lane, const VV* x, VV* q, int64_t& row, VV& qn) const {
        int u, d;
        if (!rc_tiles(unit, lane, u, d)) return false;
        row = (int64_t)u * D_dn + d;
        const VV hs = hops_v(hop_up + u, D_up, x + d, D_dn, D_up);
        qn = q[row];
        qn.x -= hs.x; qn.y -= hs.y;
        q[row] = qn;
        return true;
    }

    template <typename VV>
    __device__ __forceinline__ bool operator()(int64_t unit, int lane, VV zs, const VV* x, int64_t& row,
                                               VV& w) const {
        using T = decltype(zs.x);
        int u, d;
        unit_rc(unit, lane, u, d);
        if (d >= D_dn) return false;
        row = (int64_t)u * D_dn + d;
        const uint32_t su = st_up[u], sd = st_dn[d];
        int cu, cp, cv;
        counts(su, sd, u, d, cu, cp, cv);
        const T diag = (T)(self_up[u] + self_dn[d] + cross[min(cu, kCross2 - 1)] +
                           cross[kCross2 + min(cp, kCross2 - 1)] + cross[2 * kCross2 + min(cv, kCross2 - 1)]);
        VV acc;
        {
            const VV xr = x[row];
            const T zr = zs.x - diag;
            acc.x = zr * xr.x - zs.y * xr.y;
            acc.y = zr * xr.y + zs.y * xr.x;
        }
        for (int sp = 0; sp < 2; ++sp) {
            const int32_t* tab = sp ? hop_up + u : hop_dn + d;
            const int64_t ts = sp ? D_up : D_dn;
            const VV* base = sp ? x + d : x + (size_t)u * D_dn;
            const int64_t stride = sp ? D_dn : 1, lim = sp ? D_up : D_dn;
            for (int j = 0; j < S2; ++j) {
                const int e = tab[(int64_t)j * ts];
                if (e < 0) break;
                if (!chk(dbg, 22, e >> 8, lim)) continue;
                const VV xv = base[(int64_t)(e >> 8) * stride];
                const T t = (T)amp[(e >> 1) & 127];
                const T c = (e & 1) ? t : -t;   // - H's element
                acc.x += c * xv.x; acc.y += c * xv.y;
            }
        }
        for (int i = 0; i < ns; ++i) {
            const int32_t mu = orb_up[(size_t)i * D_up + u], md = orb_dn[(size_t)i * D_dn + d];
            if (mu < 0 || md < 0) continue;
            const int tu = mu >> 1, td = md >> 1;
            if (!chk(dbg, 23, tu, D_up) || !chk(dbg, 24, td, D_dn)) continue;
            const VV xv = x[(size_t)tu * D_dn + td];
            const T c = -(T)((mu & 1) != (md & 1) ? J : Jp);
            acc.x += c * xv.x; acc.y += c * xv.y;
        }
        w = acc;
        return true;
    }
};

template <typename R>
static ApplyHubbard2<R> make_apply2(const Hubbard& hb) {
    ApplyHubbard2<R> ap;
    const size_t D = hb.Dmax;
    ap.st_up = hb.d_states;
    ap.st_dn = hb.d_states + D;
    ap.hop_up = hb.d_hop2;
    ap.hop_dn = hb.d_hop2 + D * hb.S2;
    ap.orb_up = hb.d_orb2;
    ap.orb_dn = hb.d_orb2 + D * hb.ns;
    ap.nib_up = hb.d_nib2;
    ap.nib_dn = hb.d_nib2 + 2 * D;
    ap.self_up = hb.d_self2;
    ap.self_dn = hb.d_self2 + D;
    ap.selff_up = hb.d_self2f;
    ap.selff_dn = hb.d_self2f + D;
    ap.amp = hb.d_amp2;
    ap.ampf = reinterpret_cast<const float4*>(hb.d_amp2f);
    ap.cross = hb.d_cross2;
    ap.crossf = hb.d_cross2f;
    ap.S2 = hb.S2; ap.ns = hb.ns; ap.D_up = hb.D_up; ap.D_dn = hb.D_dn;
    ap.J = hb.J; ap.Jp = hb.Jp;
    ap.Jh = (float)(-hb.J); ap.Jl = (float)(-hb.J - (double)ap.Jh);
    ap.Ph = (float)(-hb.Jp); ap.Pl = (float)(-hb.Jp - (double)ap.Ph);
    ap.n = (int64_t)hb.D_up * hb.D_dn;
    ap.dbg = nullptr;
    return ap;
}

int hubbard2_max_ctas(const Hubbard& hb, int prec, int num_sms, size_t dyn_smem) {
    int nb = 0;
    cudaError_t e =
        prec == SCOCG_MIXED
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<float, ApplyHubbard2<float>>, kBlock,
                                                            dyn_smem)
        : prec == SCOCG_MIXED_DF
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<DF, ApplyHubbard2<float>>, kBlock,
                                                            dyn_smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<double, ApplyHubbard2<double>>,
                                                            kBlock, dyn_smem);
    (void)hb;
    return e == cudaSuccess ? nb * num_sms : 0;
}

template <typename R>
cudaError_t hubbard2_launch_solve(const SolveArgs<R>& a, const Hubbard& hb, int grid, cudaStream_t st) {
    using W = typename ValT<R>::T;
    ApplyHubbard2<W> ap = make_apply2<W>(hb);
    ap.dbg = a.dbg;
    void* args[] = {(void*)&a, (void*)&ap};
    const size_t smem = a.Xf ? (size_t)a.K * kFullSmem : 0;
    // a continuation of a stopped solve runs its own instantiation
    const void* kern = a.resume ? (const void*)cocg_persistent<R, ApplyHubbard2<W>, true>
                                : (const void*)cocg_persistent<R, ApplyHubbard2<W>, false>;
    if (smem > 0)   // above the 48 KB default together with the static part
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kBlock), args, smem, st);
}
template cudaError_t hubbard2_launch_solve<double>(const SolveArgs<double>&, const Hubbard&, int, cudaStream_t);
template cudaError_t hubbard2_launch_solve<float>(const SolveArgs<float>&, const Hubbard&, int, cudaStream_t);
template cudaError_t hubbard2_launch_solve<DF>(const SolveArgs<DF>&, const Hubbard&, int, cudaStream_t);

template <typename VV, class Apply>
__global__ void __launch_bounds__(256) k_hub2_apply(Apply ap, int64_t nunits, VV zs, const VV* x, VV* y) {
    const int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (u >= nunits) return;
    int64_t row;
    VV w;
    if (ap(u, threadIdx.x & 31, zs, x, row, w)) y[row] = w;
}

cudaError_t hubbard2_apply(const Hubbard& hb, int prec, double2 z, const void* x, void* y, cudaStream_t st) {
    const unsigned blocks = (unsigned)((hb.nunits * 32 + 255) / 256);
    if (prec == SCOCG_MIXED)
        k_hub2_apply<float2><<<blocks, 256, 0, st>>>(make_apply2<float>(hb), hb.nunits,
                                                     make_float2((float)z.x, (float)z.y), (const float2*)x,
                                                     (float2*)y);
    else if (prec == SCOCG_MIXED_DF)
        k_hub2_apply<float4><<<blocks, 256, 0, st>>>(make_apply2<float>(hb), hb.nunits, df_from(z), (const float4*)x,
                                                     (float4*)y);
    else
        k_hub2_apply<double2><<<blocks, 256, 0, st>>>(make_apply2<double>(hb), hb.nunits, z, (const double2*)x,
                                                      (double2*)y);
    return cudaGetLastError();
}

// Real FP64 operator of the ground-state iteration, y = (H - sigma) x - beta
// x_prev with the block's partial of x^T y (same contract as the ring's), in
// the two passes of the solve's phase A: pass 1 visits the units row-major
// (the CTAs share the rows x[u][:] of the down hops and the joint moves),
// pass 2 tile-major (the CTAs share the column tiles x[:][tile] of the up
// hops) and forms the partials.
__device__ __forceinline__ double hop_sum_real(const double* amp, int S2, const int32_t* tab, int64_t ts,
                                               const double* base, int64_t stride) {
    double hx = 0.0;
    for (int j = 0; j < S2; ++j) {
        const int e = tab[(int64_t)j * ts];
        if (e < 0) break;
        const double t = amp[(e >> 1) & 127];
        hx = fma((e & 1) ? -t : t, base[(int64_t)(e >> 8) * stride], hx);
    }
    return hx;
}

__global__ void __launch_bounds__(kVecBlock) k_hub2_hx1(ApplyHubbard2<double> ap, int64_t nunits, const double* x,
                                                        double* y, const double* xprev, const double* beta,
                                                        double sigma, const int* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)kVecBlock + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kVecBlock) >> 5;
    const double bp = (xprev && beta) ? *beta : 0.0;
    for (int64_t unit = w0; unit < nunits; unit += nw) {
        int u, d;
        if (!ap.rc_rows(unit, lane, u, d)) continue;
        const int64_t row = (int64_t)u * ap.D_dn + d;
        const uint32_t su = ap.st_up[u], sd = ap.st_dn[d];
        int cu, cp, cv;
        ap.counts(su, sd, u, d, cu, cp, cv);
        const double diag = ap.self_up[u] + ap.self_dn[d] + ap.cross[min(cu, kCross2 - 1)] +
                            ap.cross[kCross2 + min(cp, kCross2 - 1)] + ap.cross[2 * kCross2 + min(cv, kCross2 - 1)];
        double hx = hop_sum_real(ap.amp, ap.S2, ap.hop_dn + d, ap.D_dn, x + (size_t)u * ap.D_dn, 1);
        for (int i = 0; i < ap.ns; ++i) {
            const int32_t mu = ap.orb_up[(size_t)i * ap.D_up + u], md = ap.orb_dn[(size_t)i * ap.D_dn + d];
            if (mu < 0 || md < 0) continue;
            hx = fma((mu & 1) != (md & 1) ? ap.J : ap.Jp, x[(size_t)(mu >> 1) * ap.D_dn + (md >> 1)], hx);
        }
        double yi = fma(diag - sigma, x[row], hx);
        if (xprev) yi = fma(-bp, xprev[row], yi);
        y[row] = yi;
    }
}

__global__ void __launch_bounds__(kVecBlock, 4) k_hub2_hx2(ApplyHubbard2<double> ap, int64_t nunits, const double* x,
                                                        double* y, const int* skip, double* part) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)kVecBlock + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kVecBlock) >> 5;
    double acc = 0.0;
    for (int64_t unit = w0; unit < nunits; unit += nw) {
        int u, d;
        if (!ap.rc_tiles(unit, lane, u, d)) continue;
        const int64_t row = (int64_t)u * ap.D_dn + d;
        const double yi = y[row] + hop_sum_real(ap.amp, ap.S2, ap.hop_up + u, ap.D_up, x + d, ap.D_dn);
        y[row] = yi;
        acc = fma(x[row], yi, acc);
    }
    block_partial(acc, part);
}

cudaError_t hubbard2_hx(const Hubbard& hb, const double* x, double* y, const double* xprev, const double* beta,
                        double sigma, const int* skip, double* part, int grid, cudaStream_t st) {
    const ApplyHubbard2<double> ap = make_apply2<double>(hb);
    k_hub2_hx1<<<grid, kVecBlock, 0, st>>>(ap, hb.nunits, x, y, xprev, beta, sigma, skip);
    k_hub2_hx2<<<grid, kVecBlock, 0, st>>>(ap, hb.nunits, x, y, skip, part);
    return cudaGetLastError();
}

}  // namespace scocg

using namespace scocg;

extern "C" int scocg_create_hubbard2(scocg_handle* out, int n_sites, int n_bonds, const int32_t* bond_i,
                                     const int32_t* bond_j, const double* bond_t, double U, double Up, double J,
                                     double Jp, double V, int n_up, int n_dn, const scocg_opts* opts,
                                     void* cuda_stream) {
    if (!out) return SCOCG_ERR_INVALID;
    *out = nullptr;
    const int M = 2 * n_sites;
    if (n_sites < 1 || n_sites > kMaxSites2 || n_bonds < 0 || n_bonds > kMaxBonds2 || (n_bonds > 0 && (!bond_i || !bond_j || !bond_t)) ||
        n_up < 0 || n_dn < 0 || n_up > M || n_dn > M)
        return SCOCG_ERR_INVALID;
    for (double v : {U, Up, J, Jp, V})
        if (!std::isfinite(v)) return SCOCG_ERR_INVALID;
    int degree[kMaxSites2] = {0};
    for (int b = 0; b < n_bonds; ++b) {
        if (bond_i[b] < 0 || bond_i[b] >= n_sites || bond_j[b] < 0 || bond_j[b] >= n_sites || bond_i[b] == bond_j[b])
            return SCOCG_ERR_INVALID;
        // the neighbour sums (A n)_i <= 2 degree_i are kept in 4-bit fields
        if (++degree[bond_i[b]] > 7 || ++degree[bond_j[b]] > 7) return SCOCG_ERR_INVALID;
        for (int q = 0; q < 4; ++q)
            if (!std::isfinite(bond_t[4 * b + q])) return SCOCG_ERR_INVALID;
    }
    const int64_t Du = binom(M, n_up), Dd = binom(M, n_dn);
    // targets are packed into 24 bits of a table entry; the vector index into 63
    if (Du >= (int64_t(1) << 23) || Dd >= (int64_t(1) << 23) || Du * Dd >= (int64_t(1) << 40)) return SCOCG_ERR_INVALID;
    scocg_ctx* h = new (std::nothrow) scocg_ctx();
    if (!h) return SCOCG_ERR_OOM;
    int st = init_ctx(h, opts, cuda_stream);
    if (st != SCOCG_OK) { h->free_all(); delete h; return st; }
    Hubbard& hb = h->hub;
    hb.model = 1;
    hb.L = M; hb.n_up = n_up; hb.n_dn = n_dn; hb.periodic = 0;
    hb.ns = n_sites; hb.nb = n_bonds;
    hb.U = U; hb.Up = Up; hb.J = J; hb.Jp = Jp; hb.V = V; hb.t = 0.0;
    hb.D_up = (int)Du; hb.D_dn = (int)Dd;
    hb.Dmax = (int)std::max(Du, Dd);
    hb.S2 = std::max(1, 8 * n_bonds);
    hb.nunits = Du * ((Dd + 31) / 32);
    h->kind = HandleKind::kHubbard;
    h->n = Du * Dd;
    h->nnz = 0;
    const size_t D = hb.Dmax;
    cudaStream_t s = h->stream;
    std::vector<int32_t> bonds(2 * std::max(n_bonds, 1), 0);
    std::vector<double> amp(4 * std::max(n_bonds, 1), 0.0);
    std::vector<float4> ampf(2 * amp.size());
    for (int b = 0; b < n_bonds; ++b) {
        bonds[2 * b] = bond_i[b]; bonds[2 * b + 1] = bond_j[b];
        for (int q = 0; q < 4; ++q) amp[4 * b + q] = bond_t[4 * b + q];
    }
    for (size_t q = 0; q < amp.size(); ++q)   // entry 2 q + sign bit: the amplitude times its sign
        for (int sg = 0; sg < 2; ++sg) {
            const double v = sg ? -amp[q] : amp[q];
            const float hi = (float)v, lo = (float)(v - (double)hi);
            ampf[2 * q + sg] = make_float4(hi, hi, lo, lo);
        }
    std::vector<double> cross(3 * kCross2);
    std::vector<float2> crossf(3 * kCross2);
    for (int c = 0; c < kCross2; ++c) {
        cross[c] = U * c; cross[kCross2 + c] = Up * c; cross[2 * kCross2 + c] = V * c;
    }
    for (size_t q = 0; q < cross.size(); ++q) {
        const float hi = (float)cross[q];
        crossf[q] = make_float2(hi, (float)(cross[q] - (double)hi));
    }
    cudaError_t e = cudaMalloc(&hb.d_states, sizeof(uint32_t) * 2 * D);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_hop2, sizeof(int32_t) * 2 * D * hb.S2);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_orb2, sizeof(int32_t) * 2 * D * n_sites);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_nib2, sizeof(uint32_t) * 2 * D * 2);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_self2, sizeof(double) * 2 * D);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_self2f, sizeof(float2) * 2 * D);
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_amp2, sizeof(double) * amp.size());
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_amp2f, sizeof(float4) * ampf.size());
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_cross2, sizeof(double) * cross.size());
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_cross2f, sizeof(float2) * cross.size());
    if (e == cudaSuccess) e = cudaMalloc(&hb.d_bonds2, sizeof(int32_t) * bonds.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.d_amp2, amp.data(), sizeof(double) * amp.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.d_amp2f, ampf.data(), sizeof(float4) * ampf.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.d_cross2, cross.data(), sizeof(double) * cross.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.d_cross2f, crossf.data(), sizeof(float2) * cross.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.d_bonds2, bonds.data(), sizeof(int32_t) * bonds.size(), cudaMemcpyHostToDevice, s);
    for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp) {
        const int Ds = sp ? hb.D_dn : hb.D_up, k = sp ? n_dn : n_up;
        k_hubbard2_tables<<<(Ds + 127) / 128, 128, 0, s>>>(n_sites, n_bonds, k, Ds, hb.d_bonds2, Up, J, V, hb.S2,
                                                           hb.d_states + sp * D, hb.d_hop2 + sp * D * hb.S2,
                                                           hb.d_orb2 + sp * D * n_sites, hb.d_nib2 + sp * D * 2,
                                                           hb.d_self2 + sp * D, hb.d_self2f + sp * D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    hb.table_bytes = (double)(hb.D_up + hb.D_dn) * (4.0 + 4.0 * hb.S2 + 4.0 * n_sites + 8.0 + 8.0);
    if (e != cudaSuccess) { st = cuda_status(e); h->free_all(); delete h; return st; }
    *out = h;
    return SCOCG_OK;
}
