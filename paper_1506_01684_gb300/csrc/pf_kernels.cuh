// pf_kernels.cuh -- sm_103a kernels of one explicit time step of the grand-potential
// phase-field model (arXiv:1506.01684, Section 2, Algorithm 1), templated on the stencil
// precision R (double or float).
//
// Layout in HBM: phi as an array of 4-word cells (AoS: one 16-byte float4 / two 16-byte
// double2 per cell), mu as 2-word cells; planes are stored in a ring (moving window): logical
// plane k lives in storage plane (k + zbase) mod nz.
//
// Both sweeps tile x-y into TX x TY columns per CTA (one thread per column) and march along z
// (the paper's z-outermost order, Section 3.3), so per-plane temperature constants are formed
// once per plane and the z-neighbours stay in registers or a shared-memory ring.  Every
// staggered face value is computed once and shared by the two cells it separates: x/y faces
// through shared memory, z faces carried in registers from one plane to the next (the
// staggered-value buffering of Section 3.3).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pf_internal.h"

namespace pf {

template <typename R>
struct Ph {
    R v[4];
};
template <typename R>
struct Mu {
    R v[2];
};

// ---------------------------------------------------------------------------------------
// loads / stores (read-only path for the source fields)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ Ph<float> ldg_ph(const Ph<float> *p)
{
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    return Ph<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Ph<double> ldg_ph(const Ph<double> *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    return Ph<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ Mu<float> ldg_mu(const Mu<float> *p)
{
    float2 a = __ldg(reinterpret_cast<const float2 *>(p));
    return Mu<float>{{a.x, a.y}};
}
__device__ __forceinline__ Mu<double> ldg_mu(const Mu<double> *p)
{
    double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    return Mu<double>{{a.x, a.y}};
}
__device__ __forceinline__ void st_ph(Ph<float> *p, const Ph<float> &x)
{
    *reinterpret_cast<float4 *>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
__device__ __forceinline__ void st_ph(Ph<double> *p, const Ph<double> &x)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(x.v[0], x.v[1]);
    q[1] = make_double2(x.v[2], x.v[3]);
}
__device__ __forceinline__ void st_mu(Mu<float> *p, const Mu<float> &x)
{
    *reinterpret_cast<float2 *>(p) = make_float2(x.v[0], x.v[1]);
}
__device__ __forceinline__ void st_mu(Mu<double> *p, const Mu<double> &x)
{
    *reinterpret_cast<double2 *>(p) = make_double2(x.v[0], x.v[1]);
}

__device__ __forceinline__ int wrapi(int x, int n)
{
    // periodic index for x >= -n (x may exceed n by several periods when n < tile width)
    x %= n;
    return x < 0 ? x + n : x;
}

// storage plane of logical plane k, with the zero-gradient mirror applied first
__device__ __forceinline__ size_t plane_off(int k, int nz, int zbase, size_t plane)
{
    int kc = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
    int s = kc + zbase;
    if (s >= nz) s -= nz;
    return (size_t)s * plane;
}

template <typename R>
__device__ __forceinline__ bool same(const Ph<R> &a, const Ph<R> &b)
{
    return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2] && a.v[3] == b.v[3];
}
// phase code of a cell: the phase index of an exactly one-hot vector (one component 1, the
// others 0), 4 for any other (mixed) cell
template <typename R>
__device__ __forceinline__ int code_of(const Ph<R> &a)
{
    const R o = R(1), z = R(0);
    if (a.v[0] == o && a.v[1] == z && a.v[2] == z && a.v[3] == z) return 0;
    if (a.v[1] == o && a.v[0] == z && a.v[2] == z && a.v[3] == z) return 1;
    if (a.v[2] == o && a.v[0] == z && a.v[1] == z && a.v[3] == z) return 2;
    if (a.v[3] == o && a.v[0] == z && a.v[1] == z && a.v[2] == z) return 3;
    return 4;
}
template <typename R>
__device__ __forceinline__ bool onehot(const Ph<R> &a)
{
    return code_of(a) < 4;
}
// c-th entry of a 4-vector held in kernel parameters, without dynamic indexing
template <typename R>
__device__ __forceinline__ R pick4(const R (&v)[4], int c)
{
    return c == 0 ? v[0] : (c == 1 ? v[1] : (c == 2 ? v[2] : v[3]));
}

// ---------------------------------------------------------------------------------------
// phi-sweep pieces (Eq. 1, Eq. 2)
// ---------------------------------------------------------------------------------------

// (da/d grad phi_a)_d on the face between L and R = L + e_d, from the face average of phi
// and the face difference (the normal component depends on no other):
//   F_a = -2 sum_{b != a} gamma_ab phibar_b (phibar_a g_b - phibar_b g_a)
template <typename R>
__device__ __forceinline__ Ph<R> face_phi(const KParams<R> &kp, const Ph<R> &L, const Ph<R> &Rr)
{
    Ph<R> F;
    if (same(L, Rr)) {
        F.v[0] = F.v[1] = F.v[2] = F.v[3] = R(0);
        return F;
    }
    R p[4], g[4];
#pragma unroll
    for (int b = 0; b < 4; b++) {
        p[b] = R(0.5) * (L.v[b] + Rr.v[b]);
        g[b] = (Rr.v[b] - L.v[b]) * kp.inv_dx;
    }
    // pair values q_ab = p_a g_b - p_b g_a (q_ba = -q_ab)
    const R q01 = p[0] * g[1] - p[1] * g[0];
    const R q02 = p[0] * g[2] - p[2] * g[0];
    const R q03 = p[0] * g[3] - p[3] * g[0];
    const R q12 = p[1] * g[2] - p[2] * g[1];
    const R q13 = p[1] * g[3] - p[3] * g[1];
    const R q23 = p[2] * g[3] - p[3] * g[2];
    const R *G2 = kp.gamma2;
    F.v[0] = R(-2) * (G2[0] * p[1] * q01 + G2[1] * p[2] * q02 + G2[2] * p[3] * q03);
    F.v[1] = R(-2) * (G2[0] * p[0] * (-q01) + G2[3] * p[2] * q12 + G2[4] * p[3] * q13);
    F.v[2] = R(-2) * (G2[1] * p[0] * (-q02) + G2[3] * p[1] * (-q12) + G2[5] * p[3] * q23);
    F.v[3] = R(-2) * (G2[2] * p[0] * (-q03) + G2[4] * p[1] * (-q13) + G2[5] * p[2] * (-q23));
    return F;
}

// Euclidean projection onto {sum = 1, phi >= 0} (reading R6): sort descending (5-comparator
// network), running sums, the largest j with s_j - (c_j - 1)/j > 0 fixes the shift theta.
template <typename R>
__device__ __forceinline__ Ph<R> project_simplex(const Ph<R> &u)
{
    R s0 = u.v[0], s1 = u.v[1], s2 = u.v[2], s3 = u.v[3], tmp;
#define PF_CS(a, b)      \
    if (a < b) {         \
        tmp = a;         \
        a = b;           \
        b = tmp;         \
    }
    PF_CS(s0, s1);
    PF_CS(s2, s3);
    PF_CS(s0, s2);
    PF_CS(s1, s3);
    PF_CS(s1, s2);
#undef PF_CS
    R theta = R(0);
    R c = s0;
    R t = c - R(1);
    if (s0 - t > R(0)) theta = t;
    c = c + s1;
    t = (c - R(1)) * R(0.5);
    if (s1 - t > R(0)) theta = t;
    c = c + s2;
    t = (c - R(1)) / R(3);
    if (s2 - t > R(0)) theta = t;
    c = c + s3;
    t = (c - R(1)) * R(0.25);
    if (s3 - t > R(0)) theta = t;
    Ph<R> o;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        R r = u.v[a] - theta;
        o.v[a] = r > R(0) ? r : R(0);
    }
    return o;
}

// Full cell update of the phi-sweep at one cell.
//   xm/xp, ym/yp, zm/zp: the six neighbours; F*: the six face terms (minus/plus side).
template <typename R>
__device__ __forceinline__ Ph<R> phi_cell(const KParams<R> &kp, const PlaneT<R> &pc, const Ph<R> &P,
                                          const Ph<R> &xm, const Ph<R> &xp, const Ph<R> &ym,
                                          const Ph<R> &yp, const Ph<R> &zm, const Ph<R> &zp,
                                          const Ph<R> &Fxm, const Ph<R> &Fxp, const Ph<R> &Fym,
                                          const Ph<R> &Fyp, const Ph<R> &Fzm, const Ph<R> &Fzp,
                                          const Mu<R> &m)
{
    const R *G2 = kp.gamma2;
    const R *G3 = kp.gamma3;
    R div[4], g[4][3];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        div[a] = (Fxp.v[a] - Fxm.v[a]) * kp.inv_dx;
        div[a] = div[a] + (Fyp.v[a] - Fym.v[a]) * kp.inv_dx;
        div[a] = div[a] + (Fzp.v[a] - Fzm.v[a]) * kp.inv_dx;
        g[a][0] = (xp.v[a] - xm.v[a]) * kp.inv_2dx;
        g[a][1] = (yp.v[a] - ym.v[a]) * kp.inv_2dx;
        g[a][2] = (zp.v[a] - zm.v[a]) * kp.inv_2dx;
    }
    const R *p = P.v;
    // da/dphi_a = 2 sum_{b != a} gamma_ab (p_a g_b - p_b g_a) . g_b, one pair at a time
    R dadp[4] = {R(0), R(0), R(0), R(0)};
    const int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {1, 2, 3, 2, 3, 3};
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const int a = PA[q], b = PB[q];
        R qa = R(0), qb = R(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            R qd = p[a] * g[b][d] - p[b] * g[a][d];  // q_ab (q_ba = -q_ab)
            qa = qa + qd * g[b][d];
            qb = qb - qd * g[a][d];
        }
        dadp[a] = dadp[a] + G2[q] * qa;
        dadp[b] = dadp[b] + G2[q] * qb;
    }
    // d omega / d phi_a
    R dom[4];
    dom[0] = kp.obst * (G2[0] * p[1] + G2[1] * p[2] + G2[2] * p[3]) +
             (G3[0] * p[1] * p[2] + G3[1] * p[1] * p[3] + G3[2] * p[2] * p[3]);
    dom[1] = kp.obst * (G2[0] * p[0] + G2[3] * p[2] + G2[4] * p[3]) +
             (G3[0] * p[0] * p[2] + G3[1] * p[0] * p[3] + G3[3] * p[2] * p[3]);
    dom[2] = kp.obst * (G2[1] * p[0] + G2[3] * p[1] + G2[5] * p[3]) +
             (G3[0] * p[0] * p[1] + G3[2] * p[0] * p[3] + G3[3] * p[1] * p[3]);
    dom[3] = kp.obst * (G2[2] * p[0] + G2[4] * p[1] + G2[5] * p[2]) +
             (G3[1] * p[0] * p[1] + G3[2] * p[0] * p[2] + G3[3] * p[1] * p[2]);
    // d psi / d phi_a = 2 p_a (psi_a - sum h_b psi_b) / sum p_b^2
    R S = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + p[3] * p[3];
    R inv_S = R(1) / S;
    R mu2 = m.v[0] * m.v[0] + m.v[1] * m.v[1];
    R psi[4], hpsi = R(0);
#pragma unroll
    for (int a = 0; a < 4; a++) {
        psi[a] = -mu2 * kp.inv4A[a] - (m.v[0] * pc.chat[a][0] + m.v[1] * pc.chat[a][1]) + pc.sT[a];
        hpsi = hpsi + p[a] * p[a] * inv_S * psi[a];
    }
    R rhs[4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        R dps = R(2) * p[a] * (psi[a] - hpsi) * inv_S;
        rhs[a] = pc.epsT * (R(2) * dadp[a] - div[a]) + pc.Toeps * dom[a] + dps;
    }
    R mean = (rhs[0] + rhs[1] + rhs[2] + rhs[3]) * R(0.25);
    Ph<R> st;
#pragma unroll
    for (int a = 0; a < 4; a++) st.v[a] = p[a] - kp.c_phi * (rhs[a] - mean);
    return project_simplex(st);
}

// ---------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------
// reciprocal: correctly rounded in both precisions (exact for 1), no full division in FP32
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// one plane-table entry (16 words) through the read-only path; the same address for every
// thread of a CTA, so the loads are broadcasts served by L1
__device__ __forceinline__ PlaneT<float> ldg_plane(const PlaneT<float> *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    PlaneT<float> t;
    float4 *o = reinterpret_cast<float4 *>(&t);
#pragma unroll
    for (int w = 0; w < 4; w++) o[w] = __ldg(q + w);
    return t;
}
__device__ __forceinline__ PlaneT<double> ldg_plane(const PlaneT<double> *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    PlaneT<double> t;
    double2 *o = reinterpret_cast<double2 *>(&t);
#pragma unroll
    for (int w = 0; w < 8; w++) o[w] = __ldg(q + w);
    return t;
}

template <typename R>
struct Chat {
    R c[4][2];
};
__device__ __forceinline__ Chat<float> ldg_chat(const PlaneT<float> *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p) + 1;  // chat starts at word 4
    Chat<float> t;
    float4 *o = reinterpret_cast<float4 *>(&t);
    o[0] = __ldg(q);
    o[1] = __ldg(q + 1);
    return t;
}
__device__ __forceinline__ Chat<double> ldg_chat(const PlaneT<double> *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p) + 2;
    Chat<double> t;
    double2 *o = reinterpret_cast<double2 *>(&t);
#pragma unroll
    for (int w = 0; w < 4; w++) o[w] = __ldg(q + w);
    return t;
}

template <typename R>
__device__ __forceinline__ bool finite4(const Ph<R> &a)
{
    return isfinite(a.v[0]) && isfinite(a.v[1]) && isfinite(a.v[2]) && isfinite(a.v[3]);
}

// Ring cell number r (0 <= r < 2 (TX + TY) + 4) of a TX x TY tile -> local (li, lj) in [-1, TX] x [-1, TY]
template <int TX, int TY>
__device__ __forceinline__ void ring_cell(int r, int &li, int &lj)
{
    constexpr int SX = TX + 2;
    if (r < SX) {
        li = r - 1;
        lj = -1;
    } else if (r < 2 * SX) {
        li = r - SX - 1;
        lj = TY;
    } else {
        const int q = r - 2 * SX;
        if (q < TY) {
            li = -1;
            lj = q;
        } else {
            li = TX;
            lj = q - TY;
        }
    }
}

// ---------------------------------------------------------------------------------------
// mu-sweep pieces (Eq. 3, Eq. 4)
// ---------------------------------------------------------------------------------------

// v = M(phibar) grad mu - J_at on one face.  nL/nR: phi^{n+1} at the two cells, oL/oR: phi^n,
// mL/mR: mu^n.  a*/b*: phi^{n+1} at the tangential neighbours of L and R in the face's two
// tangential directions (the D3C19 stencil): face gradient component (L+e - L-e + R+e - R-e)/(4 dx).
// tf: plane-table entry of the face's temperature (read only where the anti-trapping current is
// evaluated).  A face between two equal one-hot cells takes the exact short form (h = phi there,
// no anti-trapping current).
template <typename R>
__device__ __forceinline__ Mu<R> face_mu_general(const KParams<R> &kp, const PlaneT<R> *__restrict__ tf,
                                                 const Ph<R> &nL, const Ph<R> &nR, const Ph<R> &oL, const Ph<R> &oR,
                                                 const Mu<R> &mL, const Mu<R> &mR, const Ph<R> &aLp,
                                                 const Ph<R> &aLm, const Ph<R> &aRp, const Ph<R> &aRm,
                                                 const Ph<R> &bLp, const Ph<R> &bLm, const Ph<R> &bRp,
                                                 const Ph<R> &bRm)
{
    Mu<R> v;
    R pb[4];
#pragma unroll
    for (int b = 0; b < 4; b++) pb[b] = R(0.5) * (nL.v[b] + nR.v[b]);
    const R S = pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2] + pb[3] * pb[3];
    const R inv_S = rcp(S);
    R h[4];
#pragma unroll
    for (int b = 0; b < 4; b++) h[b] = pb[b] * pb[b] * inv_S;
    const R M = kp.DinvA[0] * h[0] + kp.DinvA[1] * h[1] + kp.DinvA[2] * h[2] + kp.DinvA[3] * h[3];
    v.v[0] = M * (mR.v[0] - mL.v[0]) * kp.inv_dx;
    v.v[1] = M * (mR.v[1] - mL.v[1]) * kp.inv_dx;
    // anti-trapping current (Eq. 4, g_a = phi_a); terms skipped per reading R9
    if (pb[3] > R(0) && (pb[0] > R(0) || pb[1] > R(0) || pb[2] > R(0))) {
        R gl[3];
        gl[0] = (nR.v[3] - nL.v[3]) * kp.inv_dx;
        gl[1] = (aLp.v[3] - aLm.v[3] + aRp.v[3] - aRm.v[3]) * kp.inv_4dx;
        gl[2] = (bLp.v[3] - bLm.v[3] + bRp.v[3] - bRm.v[3]) * kp.inv_4dx;
        const R gl2 = gl[0] * gl[0] + gl[1] * gl[1] + gl[2] * gl[2];
        if (gl2 > kp.grad_thr) {
            const Chat<R> ch = ldg_chat(tf);
            const R nl = sqrt(gl2);
            const R mb0 = R(0.5) * (mL.v[0] + mR.v[0]);
            const R mb1 = R(0.5) * (mL.v[1] + mR.v[1]);
            const R cl0 = mb0 * kp.inv2A[3] + ch.c[3][0];
            const R cl1 = mb1 * kp.inv2A[3] + ch.c[3][1];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (!(pb[a] > R(0))) continue;
                R ga[3];
                ga[0] = (nR.v[a] - nL.v[a]) * kp.inv_dx;
                ga[1] = (aLp.v[a] - aLm.v[a] + aRp.v[a] - aRm.v[a]) * kp.inv_4dx;
                ga[2] = (bLp.v[a] - bLm.v[a] + bRp.v[a] - bRm.v[a]) * kp.inv_4dx;
                const R ga2 = ga[0] * ga[0] + ga[1] * ga[1] + ga[2] * ga[2];
                if (!(ga2 > kp.grad_thr)) continue;
                const R na = sqrt(ga2);
                const R ndot = (ga[0] * gl[0] + ga[1] * gl[1] + ga[2] * gl[2]) / (na * nl);
                const R pdot = R(0.5) * ((nL.v[a] - oL.v[a]) + (nR.v[a] - oR.v[a])) * kp.inv_dt;
                const R pref = kp.at_pref * (pb[a] * h[3] / sqrt(pb[a] * pb[3])) * pdot * ndot;
                const R dc0 = cl0 - (mb0 * kp.inv2A[a] + ch.c[a][0]);
                const R dc1 = cl1 - (mb1 * kp.inv2A[a] + ch.c[a][1]);
                const R nd = ga[0] / na;  // normal component: the face direction is component 0
                v.v[0] = v.v[0] - pref * dc0 * nd;
                v.v[1] = v.v[1] - pref * dc1 * nd;
            }
        }
    }
    return v;
}

// v = M(phibar) grad mu - J_at on one face.  nL/nR: phi^{n+1} at the two cells, oL/oR: phi^n,
// mL/mR: mu^n.  a*/b*: phi^{n+1} at the tangential neighbours of L and R in the face's two
// tangential directions (the D3C19 stencil): face gradient component (L+e - L-e + R+e - R-e)/(4 dx).
// tf: plane-table entry of the face's temperature (read only where the anti-trapping current is
// evaluated).  A face between two equal one-hot cells takes the exact short form (h = phi there,
// no anti-trapping current).
template <typename R>
__device__ __forceinline__ Mu<R> face_mu(const KParams<R> &kp, const PlaneT<R> *__restrict__ tf, const Ph<R> &nL,
                                         const Ph<R> &nR, const Ph<R> &oL, const Ph<R> &oR, const Mu<R> &mL,
                                         const Mu<R> &mR, const Ph<R> &aLp, const Ph<R> &aLm,
                                         const Ph<R> &aRp, const Ph<R> &aRm, const Ph<R> &bLp,
                                         const Ph<R> &bLm, const Ph<R> &bRp, const Ph<R> &bRm)
{
    if (same(nL, nR) && onehot(nL)) {
        Mu<R> v;
        const R M = kp.DinvA[0] * nL.v[0] + kp.DinvA[1] * nL.v[1] + kp.DinvA[2] * nL.v[2] + kp.DinvA[3] * nL.v[3];
        v.v[0] = M * (mR.v[0] - mL.v[0]) * kp.inv_dx;
        v.v[1] = M * (mR.v[1] - mL.v[1]) * kp.inv_dx;
        return v;
    }
    return face_mu_general(kp, tf, nL, nR, oL, oR, mL, mR, aLp, aLm, aRp, aRm, bLp, bLm, bRp, bRm);
}

// mu update at one cell (Eq. 3, reading R10):
//   mu^{n+1} = mu^n + [dt div v - sum_a c^a(mu^n,T)(h_a(new) - h_a(old)) - sum_a h_a(new) kT_a dT] / chi
// A cell whose phi did not change and is one-hot takes the exact short form (h = phi, no
// phase-change source).
template <typename R>
__device__ __forceinline__ Mu<R> mu_cell(const KParams<R> &kp, const PlaneT<R> *__restrict__ tc, const Ph<R> &nP,
                                         const Ph<R> &oP, const Mu<R> &m, R div0, R div1)
{
    R hN[4];
    R dphi0 = R(0), dphi1 = R(0);
    if (same(nP, oP) && onehot(nP)) {
#pragma unroll
        for (int a = 0; a < 4; a++) hN[a] = nP.v[a];
    } else {
        R hO[4];
        const R iSN = rcp(nP.v[0] * nP.v[0] + nP.v[1] * nP.v[1] + nP.v[2] * nP.v[2] + nP.v[3] * nP.v[3]);
        const R iSO = rcp(oP.v[0] * oP.v[0] + oP.v[1] * oP.v[1] + oP.v[2] * oP.v[2] + oP.v[3] * oP.v[3]);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            hN[a] = nP.v[a] * nP.v[a] * iSN;
            hO[a] = oP.v[a] * oP.v[a] * iSO;
        }
        const Chat<R> ch = ldg_chat(tc);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const R dh = hN[a] - hO[a];
            dphi0 = dphi0 + (m.v[0] * kp.inv2A[a] + ch.c[a][0]) * dh;
            dphi1 = dphi1 + (m.v[1] * kp.inv2A[a] + ch.c[a][1]) * dh;
        }
    }
    R chi = R(0), dT0 = R(0), dT1 = R(0);
#pragma unroll
    for (int a = 0; a < 4; a++) {
        chi = chi + hN[a] * kp.inv2A[a];
        dT0 = dT0 + hN[a] * kp.kT[a][0];
        dT1 = dT1 + hN[a] * kp.kT[a][1];
    }
    const R src0 = kp.dt * div0 - dphi0 - dT0 * kp.dTstep;
    const R src1 = kp.dt * div1 - dphi1 - dT1 * kp.dTstep;
    const R ichi = rcp(chi);
    Mu<R> o;
    o.v[0] = m.v[0] + src0 * ichi;
    o.v[1] = m.v[1] + src1 * ichi;
    return o;
}

// ---------------------------------------------------------------------------------------
// phi-sweep kernel: phi^{n+1} = Proj(phi^n - dt/(tau eps) (rhs - mean rhs))   (Eq. 1, Eq. 2)
//
// One barrier per plane.  Iteration p does, between two barriers:
//   C(p)   the cell update of plane p (faces of plane p from shared memory, z faces in registers),
//   B(p+1) the x/y face terms of plane p+1 (written to the other face buffer) and its z face,
//   A(p+3) the store of plane p+3 (loaded into registers during the previous iteration) into a
//          4-plane shared ring, and the loads of plane p+4.
// Each thread loads its own column and, for the first 2(TX+TY)+4 threads, one halo cell; the
// wrapped (periodic) column offsets are computed once.
// ---------------------------------------------------------------------------------------
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) phi_sweep_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi,
                                                          const Mu<R> *__restrict__ mu,
                                                          Ph<R> *__restrict__ phi_out,
                                                          const DevState *__restrict__ st,
                                                          const PlaneT<R> *__restrict__ tab)
{
    constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2, SN = SX * SY, NR = SN - NT;
    constexpr int FX = TY * (TX + 1), FY = (TY + 1) * TX;
    static_assert(NR <= NT, "one halo cell per thread at most");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ph<R> *sP = reinterpret_cast<Ph<R> *>(smem_raw);  // [4][SN]
    Ph<R> *sFx = sP + 4 * SN;                          // [2][FX]
    Ph<R> *sFy = sFx + 2 * FX;                         // [2][FY]
    Mu<R> *sMu = reinterpret_cast<Mu<R> *>(sFy + 2 * FY);  // [4][NT]: own-column mu

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const bool valid = i0 + tx < nx && j0 + ty < ny;
    const int z0 = blockIdx.z * kp.zchunk;
    const int z1 = min(z0 + kp.zchunk, nz);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;

    const int s0 = (ty + 1) * SX + (tx + 1);
    const int col0 = wrapi(j0 + ty, ny) * nx + wrapi(i0 + tx, nx);
    int s1 = -1, col1 = 0;
    if (tid < NR) {
        int li, lj;
        ring_cell<TX, TY>(tid, li, lj);
        s1 = (lj + 1) * SX + (li + 1);
        col1 = wrapi(j0 + lj, ny) * nx + wrapi(i0 + li, nx);
    }
    // extra faces: the top y face of column tx (warp 0), the right x face of row lane (warp 1)
    const bool xtra_y = ty == 0;
    const bool xtra_x = ty == 1 % TY && tx < TY;

    Ph<R> pf0, pf1;
    Mu<R> pfm;
    auto prefetch = [&](int k) {
        const size_t b = plane_off(k, nz, zbase, plane);
        pf0 = ldg_ph(phi + b + col0);
        pfm = ldg_mu(mu + b + col0);
        if (s1 >= 0) pf1 = ldg_ph(phi + b + col1);
    };
    auto commit = [&](int k) {
        Ph<R> *d = sP + (k & 3) * SN;
        d[s0] = pf0;
        if (s1 >= 0) d[s1] = pf1;
        sMu[(k & 3) * NT + tid] = pfm;
    };
    auto S = [&](int k, int li, int lj) -> const Ph<R> & { return sP[(k & 3) * SN + (lj + 1) * SX + (li + 1)]; };
    // x/y face terms of plane q and the z face (q, q+1) of this column
    auto faces = [&](int q, Ph<R> &Fz) {
        Ph<R> *fx = sFx + (q & 1) * FX;
        Ph<R> *fy = sFy + (q & 1) * FY;
        fx[ty * (TX + 1) + tx] = face_phi(kp, S(q, tx - 1, ty), S(q, tx, ty));
        fy[ty * TX + tx] = face_phi(kp, S(q, tx, ty - 1), S(q, tx, ty));
        if (xtra_y) fy[TY * TX + tx] = face_phi(kp, S(q, tx, TY - 1), S(q, tx, TY));
        if (xtra_x) fx[tx * (TX + 1) + TX] = face_phi(kp, S(q, TX - 1, tx), S(q, TX, tx));
        Fz = face_phi(kp, S(q, tx, ty), S(q + 1, tx, ty));
    };

    // prologue: planes z0-1 .. z0+2 in the ring, faces of plane z0
    for (int k = z0 - 1; k <= z0 + 2; k++) {
        prefetch(k);
        commit(k);
    }
    __syncthreads();
    Ph<R> pm = S(z0 - 1, tx, ty), pc = S(z0, tx, ty), pn = S(z0 + 1, tx, ty);
    Ph<R> Fz_prev = face_phi(kp, pm, pc), Fz_cur;
    faces(z0, Fz_cur);
    prefetch(z0 + 3);
    __syncthreads();

    for (int p = z0; p < z1; ++p) {
        // C(p)
        {
            const Ph<R> xm = S(p, tx - 1, ty), xp = S(p, tx + 1, ty);
            const Ph<R> ym = S(p, tx, ty - 1), yp = S(p, tx, ty + 1);
            const bool bulk = onehot(pc) && same(pc, xm) && same(pc, xp) && same(pc, ym) && same(pc, yp) &&
                              same(pc, pm) && same(pc, pn);
            Ph<R> out = pc;
            // bulk cells (one-hot, all six neighbours equal) are fixed points of the step; a warp
            // whose cells are all bulk skips the cell terms (the shortcuts of Section 3.3)
            if (!__all_sync(0xffffffffu, bulk)) {
                const Ph<R> *fx = sFx + (p & 1) * FX;
                const Ph<R> *fy = sFy + (p & 1) * FY;
                const PlaneT<R> T = ldg_plane(tab + p);
                out = phi_cell(kp, T, pc, xm, xp, ym, yp, pm, pn, fx[ty * (TX + 1) + tx], fx[ty * (TX + 1) + tx + 1],
                               fy[ty * TX + tx], fy[(ty + 1) * TX + tx], Fz_prev, Fz_cur, sMu[(p & 3) * NT + tid]);
            }
            if (valid) st_ph(phi_out + plane_off(p, nz, zbase, plane) + col0, out);
        }
        // B(p+1), A(p+3)
        Ph<R> Fz_next = Fz_cur;
        Ph<R> pnn = pn;
        if (p + 1 < z1) {
            faces(p + 1, Fz_next);
            pnn = S(p + 2, tx, ty);
        }
        commit(p + 3);
        prefetch(p + 4);
        __syncthreads();
        pm = pc;
        pc = pn;
        pn = pnn;
        Fz_prev = Fz_cur;
        Fz_cur = Fz_next;
    }
}

// ---------------------------------------------------------------------------------------
// mu-sweep kernel: mu^{n+1} from mu^n, phi^n, phi^{n+1}   (Eq. 3, Eq. 4), with the FP64
// per-CTA partial sums of the window trigger and the non-finite check in its epilogue.
//
// One barrier per plane, as in the phi-sweep: iteration p does C(p) (cell update of plane p),
// B(p+1) (x/y face fluxes of plane p+1 and the z face (p+1, p+2)), A(p+3) (store of plane p+3,
// loads of plane p+4).  phi^{n+1} sits in a 4-plane shared ring (the faces of plane q read planes
// q-1..q+1), phi^n and mu^n in 3-plane rings; the cell update reads its own values from registers.
// ---------------------------------------------------------------------------------------
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) mu_sweep_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi_old,
                                                         const Ph<R> *__restrict__ phi_new,
                                                         const Mu<R> *__restrict__ mu,
                                                         Mu<R> *__restrict__ mu_out,
                                                         const DevState *__restrict__ st,
                                                         const PlaneT<R> *__restrict__ tab,
                                                         Partial *__restrict__ partials)
{
    constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2, SN = SX * SY, NR = SN - NT;
    constexpr int FX = TY * (TX + 1), FY = (TY + 1) * TX;
    static_assert(NR <= NT, "one halo cell per thread at most");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ph<R> *sN = reinterpret_cast<Ph<R> *>(smem_raw);  // [4][SN] phi^{n+1}
    Ph<R> *sO = sN + 4 * SN;                           // [3][SN] phi^n
    Mu<R> *sM = reinterpret_cast<Mu<R> *>(sO + 3 * SN);  // [3][SN] mu^n
    Mu<R> *sVx = sM + 3 * SN;                          // [2][FX]
    Mu<R> *sVy = sVx + 2 * FX;                         // [2][FY]
    __shared__ double red[NT / 32][2];

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const bool valid = i0 + tx < nx && j0 + ty < ny;
    const int z0 = blockIdx.z * kp.zchunk;
    const int z1 = min(z0 + kp.zchunk, nz);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;

    const int s0 = (ty + 1) * SX + (tx + 1);
    const int col0 = wrapi(j0 + ty, ny) * nx + wrapi(i0 + tx, nx);
    int s1 = -1, col1 = 0;
    if (tid < NR) {
        int li, lj;
        ring_cell<TX, TY>(tid, li, lj);
        s1 = (lj + 1) * SX + (li + 1);
        col1 = wrapi(j0 + lj, ny) * nx + wrapi(i0 + li, nx);
    }
    const bool xtra_y = ty == 0;
    const bool xtra_x = ty == 1 % TY && tx < TY;

    Ph<R> pfN0, pfN1, pfO0, pfO1;
    Mu<R> pfM0, pfM1;
    auto mod3 = [](int k) { return (k + 3) % 3; };  // k >= -3
    auto prefetch = [&](int k) {
        const size_t b = plane_off(k, nz, zbase, plane);
        pfN0 = ldg_ph(phi_new + b + col0);
        pfO0 = ldg_ph(phi_old + b + col0);
        pfM0 = ldg_mu(mu + b + col0);
        if (s1 >= 0) {
            pfN1 = ldg_ph(phi_new + b + col1);
            pfO1 = ldg_ph(phi_old + b + col1);
            pfM1 = ldg_mu(mu + b + col1);
        }
    };
    auto commitN = [&](int k) {
        Ph<R> *d = sN + (k & 3) * SN;
        d[s0] = pfN0;
        if (s1 >= 0) d[s1] = pfN1;
    };
    auto commitOM = [&](int k) {
        const int o = mod3(k) * SN;
        sO[o + s0] = pfO0;
        sM[o + s0] = pfM0;
        if (s1 >= 0) {
            sO[o + s1] = pfO1;
            sM[o + s1] = pfM1;
        }
    };
    auto N = [&](int k, int li, int lj) -> const Ph<R> & { return sN[(k & 3) * SN + (lj + 1) * SX + (li + 1)]; };
    auto O = [&](int k, int li, int lj) -> const Ph<R> & { return sO[mod3(k) * SN + (lj + 1) * SX + (li + 1)]; };
    auto Mm = [&](int k, int li, int lj) -> const Mu<R> & { return sM[mod3(k) * SN + (lj + 1) * SX + (li + 1)]; };

    // x face (li | li+1) and y face (lj | lj+1) of plane q
    auto xface = [&](int q, int li, int lj) -> Mu<R> {
        return face_mu(kp, tab + q, N(q, li, lj), N(q, li + 1, lj), O(q, li, lj), O(q, li + 1, lj), Mm(q, li, lj),
                       Mm(q, li + 1, lj), N(q, li, lj + 1), N(q, li, lj - 1), N(q, li + 1, lj + 1),
                       N(q, li + 1, lj - 1), N(q + 1, li, lj), N(q - 1, li, lj), N(q + 1, li + 1, lj),
                       N(q - 1, li + 1, lj));
    };
    auto yface = [&](int q, int li, int lj) -> Mu<R> {
        return face_mu(kp, tab + q, N(q, li, lj), N(q, li, lj + 1), O(q, li, lj), O(q, li, lj + 1), Mm(q, li, lj),
                       Mm(q, li, lj + 1), N(q, li + 1, lj), N(q, li - 1, lj), N(q, li + 1, lj + 1),
                       N(q, li - 1, lj + 1), N(q + 1, li, lj), N(q - 1, li, lj), N(q + 1, li, lj + 1),
                       N(q - 1, li, lj + 1));
    };
    // z face (q | q+1) of this thread's column; zero at the mirror boundaries
    auto zface = [&](int q) -> Mu<R> {
        if (q < 0 || q >= nz - 1) {
            Mu<R> v;
            v.v[0] = v.v[1] = R(0);
            return v;
        }
        return face_mu(kp, tab + nz + q, N(q, tx, ty), N(q + 1, tx, ty), O(q, tx, ty), O(q + 1, tx, ty),
                       Mm(q, tx, ty), Mm(q + 1, tx, ty), N(q, tx + 1, ty), N(q, tx - 1, ty), N(q + 1, tx + 1, ty),
                       N(q + 1, tx - 1, ty), N(q, tx, ty + 1), N(q, tx, ty - 1), N(q + 1, tx, ty + 1),
                       N(q + 1, tx, ty - 1));
    };
    auto faces = [&](int q) {
        Mu<R> *vx = sVx + (q & 1) * FX;
        Mu<R> *vy = sVy + (q & 1) * FY;
        vx[ty * (TX + 1) + tx] = xface(q, tx - 1, ty);
        vy[ty * TX + tx] = yface(q, tx, ty - 1);
        if (xtra_y) vy[TY * TX + tx] = yface(q, tx, TY - 1);
        if (xtra_x) vx[tx * (TX + 1) + TX] = xface(q, TX - 1, tx);
    };

    double liq_def = 0.0;
    bool bad = false;

    // prologue: phi^{n+1} planes z0-1..z0+2, phi^n / mu^n planes z0-1..z0+1, then the z face below
    // z0, the faces of plane z0, and the phi^n / mu^n plane z0+2 once plane z0-1 is no longer read
    for (int k = z0 - 1; k <= z0 + 1; k++) {
        prefetch(k);
        commitN(k);
        commitOM(k);
    }
    prefetch(z0 + 2);
    commitN(z0 + 2);
    __syncthreads();
    Mu<R> Vz_prev = zface(z0 - 1);
    faces(z0);
    Mu<R> Vz_cur = zface(z0);
    Ph<R> ownN = N(z0, tx, ty), ownO = O(z0, tx, ty);
    Mu<R> ownM = Mm(z0, tx, ty);
    __syncthreads();
    commitOM(z0 + 2);
    prefetch(z0 + 3);
    __syncthreads();

    for (int p = z0; p < z1; ++p) {
        // C(p)
        {
            const Mu<R> *vx = sVx + (p & 1) * FX;
            const Mu<R> *vy = sVy + (p & 1) * FY;
            const Mu<R> vxm = vx[ty * (TX + 1) + tx], vxp = vx[ty * (TX + 1) + tx + 1];
            const Mu<R> vym = vy[ty * TX + tx], vyp = vy[(ty + 1) * TX + tx];
            R div0 = (vxp.v[0] - vxm.v[0]) * kp.inv_dx;
            R div1 = (vxp.v[1] - vxm.v[1]) * kp.inv_dx;
            div0 = div0 + (vyp.v[0] - vym.v[0]) * kp.inv_dx;
            div1 = div1 + (vyp.v[1] - vym.v[1]) * kp.inv_dx;
            div0 = div0 + (Vz_cur.v[0] - Vz_prev.v[0]) * kp.inv_dx;
            div1 = div1 + (Vz_cur.v[1] - Vz_prev.v[1]) * kp.inv_dx;
            const Mu<R> out = mu_cell(kp, tab + p, ownN, ownO, ownM, div0, div1);
            if (valid) {
                st_mu(mu_out + plane_off(p, nz, zbase, plane) + col0, out);
                liq_def += 1.0 - (double)ownN.v[3];
                bad = bad || !isfinite(out.v[0]) || !isfinite(out.v[1]) || !finite4(ownN);
            }
        }
        // B(p+1), A(p+3)
        Mu<R> Vz_next = Vz_cur;
        if (p + 1 < z1) {
            faces(p + 1);
            Vz_next = zface(p + 1);
            ownN = N(p + 1, tx, ty);
            ownO = O(p + 1, tx, ty);
            ownM = Mm(p + 1, tx, ty);
        }
        commitN(p + 3);
        commitOM(p + 3);
        prefetch(p + 4);
        __syncthreads();
        Vz_prev = Vz_cur;
        Vz_cur = Vz_next;
    }

    // FP64 per-CTA partials (fixed order: lanes by a shuffle tree, then warps in order)
    double badv = bad ? 1.0 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        liq_def += __shfl_down_sync(0xffffffffu, liq_def, o);
        badv += __shfl_down_sync(0xffffffffu, badv, o);
    }
    const int w = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        red[w][0] = liq_def;
        red[w][1] = badv;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < NT / 32; q++) {
            a += red[q][0];
            b += red[q][1];
        }
        const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[bid].liq_deficit = a;
        partials[bid].nonfinite = b;
    }
}

// ---------------------------------------------------------------------------------------
// fused step kernel: phi^{n+1} and mu^{n+1} in one pass (48 algorithmic bytes per FP32 cell:
// read phi^n and mu^n, write phi^{n+1} and mu^{n+1})
//
// Algorithm 1 orders the two sweeps with a full-field barrier because the mu-sweep reads
// phi^{n+1} on its D3C19 neighbourhood.  Here each CTA recomputes phi^{n+1} itself on its tile
// plus a one-cell ring (from phi^n on a two-cell ring), so the mu update follows in the same
// z-march without phi^{n+1} ever going back to HBM and being read again.  Per plane q (four
// barriers):
//   S0  store phi^n(q+2) [2-ring] and mu^n(q+2) [1-ring] (loaded during the previous plane)
//       into 3-plane shared rings, with each cell's phase code; load plane q+3 into registers
//   S1  phi face terms of plane q+1 on the 1-ring region; z face terms of the thread's cells
//   S2  phi^{n+1}(q+1) on the 1-ring region (tile cells also go to HBM)
//   S3  mu face fluxes of plane q on the tile, z flux (q, q+1) of the thread's column
//   S4  mu^{n+1}(q) of the thread's column, FP64 partial sums
// Phase codes (phase index of an exactly one-hot cell, 4 otherwise) turn the bulk tests of
// faces and cells into two byte compares; the short forms they select are exact.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ Mu<R> face_mu_coded(const KParams<R> &kp, const PlaneT<R> *__restrict__ tf, int cL, int cR,
                                               const Ph<R> &nL, const Ph<R> &nR, const Ph<R> &oL, const Ph<R> &oR,
                                               const Mu<R> &mL, const Mu<R> &mR, const Ph<R> &aLp,
                                               const Ph<R> &aLm, const Ph<R> &aRp, const Ph<R> &aRm,
                                               const Ph<R> &bLp, const Ph<R> &bLm, const Ph<R> &bRp,
                                               const Ph<R> &bRm)
{
    if (cL == cR && cL < 4) {
        Mu<R> v;
        const R M = pick4(kp.DinvA, cL);
        v.v[0] = M * (mR.v[0] - mL.v[0]) * kp.inv_dx;
        v.v[1] = M * (mR.v[1] - mL.v[1]) * kp.inv_dx;
        return v;
    }
    return face_mu_general(kp, tf, nL, nR, oL, oR, mL, mR, aLp, aLm, aRp, aRm, bLp, bLm, bRp, bRm);
}

template <typename R>
__device__ __forceinline__ Mu<R> mu_cell_coded(const KParams<R> &kp, const PlaneT<R> *__restrict__ tc, int cN,
                                               int cO, const Ph<R> &nP, const Ph<R> &oP, const Mu<R> &m, R div0,
                                               R div1)
{
    if (cN == cO && cN < 4) {
        // phi unchanged and one-hot: h = phi, no phase-change source (exactly the general form)
        const R chi = pick4(kp.inv2A, cN);
        const R kT0[4] = {kp.kT[0][0], kp.kT[1][0], kp.kT[2][0], kp.kT[3][0]};
        const R kT1[4] = {kp.kT[0][1], kp.kT[1][1], kp.kT[2][1], kp.kT[3][1]};
        const R src0 = kp.dt * div0 - R(0) - pick4(kT0, cN) * kp.dTstep;
        const R src1 = kp.dt * div1 - R(0) - pick4(kT1, cN) * kp.dTstep;
        const R ichi = rcp(chi);
        Mu<R> o;
        o.v[0] = m.v[0] + src0 * ichi;
        o.v[1] = m.v[1] + src1 * ichi;
        return o;
    }
    return mu_cell(kp, tc, nP, oP, m, div0, div1);
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) fused_step_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi,
                                                           const Mu<R> *__restrict__ mu,
                                                           Ph<R> *__restrict__ phi_out, Mu<R> *__restrict__ mu_out,
                                                           const DevState *__restrict__ st,
                                                           const PlaneT<R> *__restrict__ tab,
                                                           Partial *__restrict__ partials)
{
    constexpr int NT = TX * TY;
    constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY, NR = SN - NT;  // tile + 1-ring
    constexpr int SX2 = TX + 4, SY2 = TY + 4, SN2 = SX2 * SY2;           // tile + 2-ring
    constexpr int PFX = (TX + 3) * (TY + 2), PFY = (TX + 2) * (TY + 3);   // phi faces of the 1-ring region
    constexpr int FX = TY * (TX + 1), FY = (TY + 1) * TX;                 // mu faces of the tile
    constexpr int L2 = (SN2 + NT - 1) / NT, L1 = (SN + NT - 1) / NT;      // load slots per thread
    static_assert(NR <= NT && L2 <= 2 && L1 <= 2, "tile too small for the slot layout");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ph<R> *sO = reinterpret_cast<Ph<R> *>(smem_raw);       // [3][SN2] phi^n
    Ph<R> *sN = sO + 3 * SN2;                                // [3][SN]  phi^{n+1}
    Ph<R> *sFx = sN + 3 * SN;                                // [PFX]
    Ph<R> *sFy = sFx + PFX;                                  // [PFY]
    Mu<R> *sM = reinterpret_cast<Mu<R> *>(sFy + PFY);        // [3][SN]  mu^n
    Mu<R> *sVx = sM + 3 * SN;                                // [FX]
    Mu<R> *sVy = sVx + FX;                                   // [FY]
    unsigned char *cO = reinterpret_cast<unsigned char *>(sVy + FY);  // [3][SN2]
    unsigned char *cN = cO + 3 * SN2;                                  // [3][SN]
    __shared__ double red[NT / 32][2];

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const bool valid = i0 + tx < nx && j0 + ty < ny;
    const int z0 = blockIdx.z * kp.zchunk;
    const int z1 = min(z0 + kp.zchunk, nz);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;
    const int col_own = wrapi(j0 + ty, ny) * nx + wrapi(i0 + tx, nx);

    auto mod3 = [](int k) { return (k + 6) % 3; };  // k >= -6
    auto io = [](int li, int lj) { return (lj + 2) * SX2 + (li + 2); };  // 2-ring layout
    auto in1 = [](int li, int lj) { return (lj + 1) * SX + (li + 1); };  // 1-ring layout

    // load slots (phi^n on the 2-ring region, mu^n on the 1-ring region), offsets computed once
    int colO[2], idxO[2], colM[2], idxM[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const int r = tid + s * NT;
        idxO[s] = r < SN2 ? r : -1;
        colO[s] = 0;
        if (r < SN2) colO[s] = wrapi(j0 + r / SX2 - 2, ny) * nx + wrapi(i0 + r % SX2 - 2, nx);
        idxM[s] = r < SN ? r : -1;
        colM[s] = 0;
        if (r < SN) colM[s] = wrapi(j0 + r / SX - 1, ny) * nx + wrapi(i0 + r % SX - 1, nx);
    }
    // the thread's phi cells on the 1-ring region: its own tile cell, and one ring cell for tid < NR
    int cli[2], clj[2];
    cli[0] = tx;
    clj[0] = ty;
    const bool has_ring = tid < NR;
    cli[1] = -1;
    clj[1] = -1;
    if (has_ring) ring_cell<TX, TY>(tid, cli[1], clj[1]);
    const bool xtra_y = ty == 0;
    const bool xtra_x = ty == 1 % TY && tx < TY;

    Ph<R> pfO[2];
    Mu<R> pfM[2];
    auto prefetch = [&](int k) {
        const size_t b = plane_off(k, nz, zbase, plane);
#pragma unroll
        for (int s = 0; s < 2; s++) {
            if (idxO[s] >= 0) pfO[s] = ldg_ph(phi + b + colO[s]);
            if (idxM[s] >= 0) pfM[s] = ldg_mu(mu + b + colM[s]);
        }
    };
    auto commit = [&](int k) {
        const int so = mod3(k);
#pragma unroll
        for (int s = 0; s < 2; s++) {
            if (idxO[s] >= 0) {
                sO[so * SN2 + idxO[s]] = pfO[s];
                cO[so * SN2 + idxO[s]] = (unsigned char)code_of(pfO[s]);
            }
            if (idxM[s] >= 0) sM[so * SN + idxM[s]] = pfM[s];
        }
    };
    auto O = [&](int k, int li, int lj) -> const Ph<R> & { return sO[mod3(k) * SN2 + io(li, lj)]; };
    auto CO = [&](int k, int li, int lj) -> int { return cO[mod3(k) * SN2 + io(li, lj)]; };
    auto N = [&](int k, int li, int lj) -> const Ph<R> & { return sN[mod3(k) * SN + in1(li, lj)]; };
    auto CN = [&](int k, int li, int lj) -> int { return cN[mod3(k) * SN + in1(li, lj)]; };
    auto Mm = [&](int k, int li, int lj) -> const Mu<R> & { return sM[mod3(k) * SN + in1(li, lj)]; };

    // S1: phi face terms of plane q on the 1-ring region (x faces li|li+1 for li in [-2, TX],
    // rows [-1, TY]; y faces lj|lj+1 for lj in [-2, TY], columns [-1, TX])
    auto phi_faces = [&](int q) {
        for (int f = tid; f < PFX + PFY; f += NT) {
            int li, lj, ri, rj;
            Ph<R> *dst;
            if (f < PFX) {
                li = f % (TX + 3) - 2;
                lj = f / (TX + 3) - 1;
                ri = li + 1;
                rj = lj;
                dst = sFx + f;
            } else {
                const int g = f - PFX;
                li = g % (TX + 2) - 1;
                lj = g / (TX + 2) - 2;
                ri = li;
                rj = lj + 1;
                dst = sFy + g;
            }
            const int a = CO(q, li, lj), b = CO(q, ri, rj);
            if (a == b && a < 4) {
                Ph<R> z;
                z.v[0] = z.v[1] = z.v[2] = z.v[3] = R(0);
                *dst = z;
            } else {
                *dst = face_phi(kp, O(q, li, lj), O(q, ri, rj));
            }
        }
    };
    auto fx_at = [&](int li, int lj) -> const Ph<R> & { return sFx[(lj + 1) * (TX + 3) + (li + 2)]; };
    auto fy_at = [&](int li, int lj) -> const Ph<R> & { return sFy[(lj + 2) * (TX + 2) + (li + 1)]; };
    auto zface_phi = [&](int q, int li, int lj) -> Ph<R> {
        // z face (q | q+1) of a 1-ring cell; equal one-hot cells give zero
        const int a = CO(q, li, lj), b = CO(q + 1, li, lj);
        if (a == b && a < 4) {
            Ph<R> z;
            z.v[0] = z.v[1] = z.v[2] = z.v[3] = R(0);
            return z;
        }
        return face_phi(kp, O(q, li, lj), O(q + 1, li, lj));
    };

    // S2 for one cell: phi^{n+1}(q) at (li, lj), given its z face terms below / above
    auto phi_new_cell = [&](int q, int li, int lj, const Ph<R> &Fzm, const Ph<R> &Fzp, bool active) -> Ph<R> {
        const int c = CO(q, li, lj);
        const bool bulk = !active || (c < 4 && CO(q, li - 1, lj) == c && CO(q, li + 1, lj) == c &&
                                      CO(q, li, lj - 1) == c && CO(q, li, lj + 1) == c && CO(q - 1, li, lj) == c &&
                                      CO(q + 1, li, lj) == c);
        Ph<R> out = O(q, li, lj);
        if (!__all_sync(0xffffffffu, bulk)) {
            if (active) {
                const PlaneT<R> T = ldg_plane(tab + q);
                out = phi_cell(kp, T, O(q, li, lj), O(q, li - 1, lj), O(q, li + 1, lj), O(q, li, lj - 1),
                               O(q, li, lj + 1), O(q - 1, li, lj), O(q + 1, li, lj), fx_at(li - 1, lj), fx_at(li, lj),
                               fy_at(li, lj - 1), fy_at(li, lj), Fzm, Fzp, Mm(q, li, lj));
            }
        }
        return out;
    };
    // S2: phi^{n+1}(q) for the thread's cells (a copy of plane nz-1 / 0 outside the domain)
    Ph<R> Fz_lo[2], Fz_hi[2];
    auto phi_new_plane = [&](int q) {
        const int sn = mod3(q) * SN;
        if (q >= 0 && q < nz) {
#pragma unroll
            for (int s = 0; s < 2; s++) {
                if (s == 1 && tid >= 96) break;  // warps 0-2 hold the ring cells
                const bool act = s == 0 || has_ring;
                const int li = cli[s], lj = clj[s];
                const Ph<R> v = phi_new_cell(q, act ? li : 0, act ? lj : 0, Fz_lo[s], Fz_hi[s], act);
                if (act) {
                    sN[sn + in1(li, lj)] = v;
                    cN[sn + in1(li, lj)] = (unsigned char)code_of(v);
                    if (s == 0 && valid && q >= z0 && q < z1) st_ph(phi_out + plane_off(q, nz, zbase, plane) + col_own, v);
                }
            }
        }
    };
    // the mirror planes -1 and nz hold copies of planes 0 and nz-1 (run after a barrier)
    auto mirror_plane = [&](int q, int from) {
        const int d = mod3(q) * SN, s0 = mod3(from) * SN;
        for (int r = tid; r < SN; r += NT) {
            sN[d + r] = sN[s0 + r];
            cN[d + r] = cN[s0 + r];
        }
    };

    // S3: mu faces of plane q (tile) and the z face (q | q+1) of this column
    auto xface = [&](int q, int li, int lj) -> Mu<R> {
        return face_mu_coded(kp, tab + q, CN(q, li, lj), CN(q, li + 1, lj), N(q, li, lj), N(q, li + 1, lj), O(q, li, lj),
                             O(q, li + 1, lj), Mm(q, li, lj), Mm(q, li + 1, lj), N(q, li, lj + 1), N(q, li, lj - 1),
                             N(q, li + 1, lj + 1), N(q, li + 1, lj - 1), N(q + 1, li, lj), N(q - 1, li, lj),
                             N(q + 1, li + 1, lj), N(q - 1, li + 1, lj));
    };
    auto yface = [&](int q, int li, int lj) -> Mu<R> {
        return face_mu_coded(kp, tab + q, CN(q, li, lj), CN(q, li, lj + 1), N(q, li, lj), N(q, li, lj + 1), O(q, li, lj),
                             O(q, li, lj + 1), Mm(q, li, lj), Mm(q, li, lj + 1), N(q, li + 1, lj), N(q, li - 1, lj),
                             N(q, li + 1, lj + 1), N(q, li - 1, lj + 1), N(q + 1, li, lj), N(q - 1, li, lj),
                             N(q + 1, li, lj + 1), N(q - 1, li, lj + 1));
    };
    auto zface_mu = [&](int q) -> Mu<R> {
        if (q < 0 || q >= nz - 1) {
            Mu<R> v;
            v.v[0] = v.v[1] = R(0);
            return v;
        }
        return face_mu_coded(kp, tab + nz + q, CN(q, tx, ty), CN(q + 1, tx, ty), N(q, tx, ty), N(q + 1, tx, ty),
                             O(q, tx, ty), O(q + 1, tx, ty), Mm(q, tx, ty), Mm(q + 1, tx, ty), N(q, tx + 1, ty),
                             N(q, tx - 1, ty), N(q + 1, tx + 1, ty), N(q + 1, tx - 1, ty), N(q, tx, ty + 1),
                             N(q, tx, ty - 1), N(q + 1, tx, ty + 1), N(q + 1, tx, ty - 1));
    };
    auto mu_faces = [&](int q) {
        sVx[ty * (TX + 1) + tx] = xface(q, tx - 1, ty);
        sVy[ty * TX + tx] = yface(q, tx, ty - 1);
        if (xtra_y) sVy[TY * TX + tx] = yface(q, tx, TY - 1);
        if (xtra_x) sVx[tx * (TX + 1) + TX] = xface(q, TX - 1, tx);
    };

    double liq_def = 0.0;
    int solid_cells = 0;
    bool bad = false;

    // ---- prologue: phi^{n+1} on planes z0-1 and z0, the z flux below z0 ----
    prefetch(z0 - 2);
    commit(z0 - 2);
    prefetch(z0 - 1);
    commit(z0 - 1);
    prefetch(z0);
    commit(z0);
    prefetch(z0 + 1);
    __syncthreads();
    phi_faces(z0 - 1);
#pragma unroll
    for (int s = 0; s < 2; s++) {
        Fz_lo[s] = zface_phi(z0 - 2, cli[s], clj[s]);
        Fz_hi[s] = zface_phi(z0 - 1, cli[s], clj[s]);
    }
    __syncthreads();
    if (z0 > 0) phi_new_plane(z0 - 1);
    __syncthreads();
    commit(z0 + 1);  // replaces plane z0-2, read for the last time above
    prefetch(z0 + 2);
    phi_faces(z0);  // plane z0 only reads plane z0 (present since the first barrier)
#pragma unroll
    for (int s = 0; s < 2; s++) Fz_lo[s] = Fz_hi[s];  // z face (z0-1 | z0)
    __syncthreads();  // plane z0+1 and the faces of plane z0 are visible
#pragma unroll
    for (int s = 0; s < 2; s++) Fz_hi[s] = zface_phi(z0, cli[s], clj[s]);
    phi_new_plane(z0);
    __syncthreads();
    if (z0 == 0) {
        mirror_plane(-1, 0);
        __syncthreads();
    }
    Mu<R> Vz_lo = zface_mu(z0 - 1);
    __syncthreads();  // plane z0-1 of phi^n / mu^n is replaced by the first commit below

    // ---- main loop over planes ----
    for (int q = z0; q < z1; ++q) {
        // S0
        commit(q + 2);
        prefetch(q + 3);
        __syncthreads();
        // S1: faces of plane q+1, z faces (q+1 | q+2)
        phi_faces(q + 1);
#pragma unroll
        for (int s = 0; s < 2; s++) {
            Fz_lo[s] = Fz_hi[s];
            Fz_hi[s] = zface_phi(q + 1, cli[s], clj[s]);
        }
        __syncthreads();
        // S2: phi^{n+1}(q+1) (a copy of plane nz-1 above the domain)
        if (q + 1 < nz) {
            phi_new_plane(q + 1);
        } else {
            const int d = mod3(q + 1) * SN, s0 = mod3(q) * SN;
            for (int r = tid; r < SN; r += NT) {
                sN[d + r] = sN[s0 + r];
                cN[d + r] = cN[s0 + r];
            }
        }
        __syncthreads();
        // S3: mu faces of plane q
        mu_faces(q);
        const Mu<R> Vz_hi = zface_mu(q);
        const Ph<R> nP = N(q, tx, ty), oP = O(q, tx, ty);
        const int cn = CN(q, tx, ty), co = CO(q, tx, ty);
        const Mu<R> mP = Mm(q, tx, ty);
        __syncthreads();
        // S4: mu^{n+1}(q)
        {
            const Mu<R> vxm = sVx[ty * (TX + 1) + tx], vxp = sVx[ty * (TX + 1) + tx + 1];
            const Mu<R> vym = sVy[ty * TX + tx], vyp = sVy[(ty + 1) * TX + tx];
            R div0 = (vxp.v[0] - vxm.v[0]) * kp.inv_dx;
            R div1 = (vxp.v[1] - vxm.v[1]) * kp.inv_dx;
            div0 = div0 + (vyp.v[0] - vym.v[0]) * kp.inv_dx;
            div1 = div1 + (vyp.v[1] - vym.v[1]) * kp.inv_dx;
            div0 = div0 + (Vz_hi.v[0] - Vz_lo.v[0]) * kp.inv_dx;
            div1 = div1 + (Vz_hi.v[1] - Vz_lo.v[1]) * kp.inv_dx;
            const Mu<R> out = mu_cell_coded(kp, tab + q, cn, co, nP, oP, mP, div0, div1);
            if (valid) {
                st_mu(mu_out + plane_off(q, nz, zbase, plane) + col_own, out);
                if (cn == 3) {
                } else if (cn < 3) {
                    solid_cells++;
                } else {
                    liq_def += 1.0 - (double)nP.v[3];
                }
                bad = bad || !isfinite(out.v[0]) || !isfinite(out.v[1]) || !finite4(nP);
            }
        }
        Vz_lo = Vz_hi;
    }

    // FP64 per-CTA partials (fixed order: lanes by a shuffle tree, then warps in order)
    liq_def += (double)solid_cells;
    double badv = bad ? 1.0 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        liq_def += __shfl_down_sync(0xffffffffu, liq_def, o);
        badv += __shfl_down_sync(0xffffffffu, badv, o);
    }
    const int w = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        red[w][0] = liq_def;
        red[w][1] = badv;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < NT / 32; q++) {
            a += red[q][0];
            b += red[q][1];
        }
        const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[bid].liq_deficit = a;
        partials[bid].nonfinite = b;
    }
}

// ---------------------------------------------------------------------------------------
// per-step bookkeeping kernels
// ---------------------------------------------------------------------------------------

// Temperature-dependent constants of one plane level zc (in planes, FP64) at time t.
template <typename R>
__device__ __forceinline__ void make_plane(const KParams<R> &kp, double zc, double t, PlaneT<R> *out)
{
    const double T = kp.T0 + kp.G * (zc * kp.dx64 - kp.v * t);  // T = T0 + G (z - v t)
    const double dT = T - kp.TE;
    PlaneT<R> c;
    c.T = (R)T;
    c.epsT = (R)(kp.eps64 * T);
    c.Toeps = (R)(T / kp.eps64);
    c.pad0 = R(0);
#pragma unroll
    for (int a = 0; a < 4; a++) {
        c.chat[a][0] = (R)(kp.cE[a][0] + kp.kT64[a][0] * dT);
        c.chat[a][1] = (R)(kp.cE[a][1] + kp.kT64[a][1] * dT);
        c.sT[a] = (R)(kp.s64[a] * dT);
    }
    *out = c;
}

// One block: reduce the mu-sweep partials in a fixed order, advance t, latch non-finite
// values, and decide the moving-window shift (reading R11).
template <typename R>
__global__ void __launch_bounds__(256) finalize_kernel(const KParams<R> kp, DevState *__restrict__ st,
                                                      const Partial *__restrict__ parts, int nparts)
{
    __shared__ double sa[256], sb[256];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 256) {
        a += parts[q].liq_deficit;
        b += parts[q].nonfinite;
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->t = st->t + kp.dt64;
        if (sb[0] > 0.0) st->nonfinite = 1;
        const double h = sa[0] / ((double)kp.nx * (double)kp.ny);
        st->h_int = h;
        int s = 0;
        if (kp.window && h >= kp.window_trigger_z) {
            s = (int)floor(h - kp.window_trigger_z) + 1;
            if (s > kp.nz - 1) s = kp.nz - 1;
            if (s < 0) s = 0;
        }
        st->shift = s;
        if (s > 0) {
            int zb = st->zbase + s;
            if (zb >= kp.nz) zb -= kp.nz;
            st->zbase = zb;
            st->off = st->off + (double)s;
            st->nshift_total += s;
        }
    }
}

// After finalize: rebuild the plane table for the new (t, offset) and fill the planes that
// entered the window (phi = liquid, mu = the previous top plane's mu).
template <typename R>
__global__ void __launch_bounds__(256) post_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                  Ph<R> *__restrict__ phi, Mu<R> *__restrict__ mu,
                                                  PlaneT<R> *__restrict__ tab)
{
    const double t = st->t, off = st->off;
    const int s = st->shift, zbase = st->zbase;
    const int nz = kp.nz;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t e = tid; e < (size_t)2 * nz; e += nth) {
        if (e < (size_t)nz)
            make_plane(kp, (double)e + off, t, tab + e);
        else
            make_plane(kp, ((double)(e - nz) + off) + 0.5, t, tab + e);
    }
    if (s > 0) {
        const size_t plane = (size_t)kp.nx * kp.ny;
        const size_t src = plane_off(nz - 1 - s, nz, zbase, plane);
        for (size_t q = tid; q < (size_t)s * plane; q += nth) {
            const int kk = nz - s + (int)(q / plane);
            const size_t c = q % plane;
            const size_t dst = plane_off(kk, nz, zbase, plane) + c;
            Ph<R> liq;
            liq.v[0] = liq.v[1] = liq.v[2] = R(0);
            liq.v[3] = R(1);
            st_ph(phi + dst, liq);
            st_mu(mu + dst, mu[src + c]);
        }
    }
}

// Voronoi nuclei (reading R13): cells with k < H take the phase of the nearest seed
// (periodic distance in x and y, cell centres at +1/2, ties to the lowest grain); liquid above.
// The distance is formed with explicitly rounded FP64 operations (no contraction), so the
// nearest-seed decision is the same in every build.
template <typename R>
__global__ void __launch_bounds__(256) init_kernel(const KParams<R> kp, Ph<R> *__restrict__ phi,
                                                  Mu<R> *__restrict__ mu, const double *__restrict__ seeds,
                                                  int n_grains, int H)
{
    const size_t plane = (size_t)kp.nx * kp.ny, n = plane * kp.nz;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / plane);
        const int j = (int)((q % plane) / kp.nx);
        const int i = (int)(q % kp.nx);
        int ph = 3;
        if (k < H && n_grains > 0) {
            int best = -1;
            double bestd = 0.0;
            for (int g = 0; g < n_grains; g++) {
                double ddx = fabs(__dadd_rn((double)i + 0.5, -seeds[4 * g + 0]));
                double ddy = fabs(__dadd_rn((double)j + 0.5, -seeds[4 * g + 1]));
                double ddz = fabs(__dadd_rn((double)k + 0.5, -seeds[4 * g + 2]));
                const double wx = __dadd_rn((double)kp.nx, -ddx), wy = __dadd_rn((double)kp.ny, -ddy);
                if (wx < ddx) ddx = wx;
                if (wy < ddy) ddy = wy;
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                if (best < 0 || d2 < bestd) {
                    best = g;
                    bestd = d2;
                }
            }
            ph = (int)seeds[4 * best + 3];
        }
        Ph<R> v;
#pragma unroll
        for (int a = 0; a < 4; a++) v.v[a] = a == ph ? R(1) : R(0);
        st_ph(phi + q, v);
        Mu<R> m;
        m.v[0] = m.v[1] = R(0);
        st_mu(mu + q, m);
    }
}

// FP64 diagnostics per logical plane (one block per plane): sum phi_a (4), solute sum c_i (2)
// with c = sum_a h_a (mu/(2 A_a) + cE_a + kT_a (T - TE)), sum (1 - phi_l), non-finite count.
template <typename R>
__global__ void __launch_bounds__(256) reduce_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                    const Ph<R> *__restrict__ phi, const Mu<R> *__restrict__ mu,
                                                    double *__restrict__ out)
{
    __shared__ double sh[8][256];
    const int k = blockIdx.x;
    const size_t plane = (size_t)kp.nx * kp.ny;
    const size_t base = plane_off(k, kp.nz, st->zbase, plane);
    const double T = kp.T0 + kp.G * (((double)k + st->off) * kp.dx64 - kp.v * st->t);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (size_t q = threadIdx.x; q < plane; q += 256) {
        const Ph<R> p = ldg_ph(phi + base + q);
        const Mu<R> m = ldg_mu(mu + base + q);
        double ph[4], S = 0.0;
        for (int a = 0; a < 4; a++) {
            ph[a] = (double)p.v[a];
            S += ph[a] * ph[a];
        }
        const double m0 = (double)m.v[0], m1 = (double)m.v[1];
        bool bad = !isfinite(m0) || !isfinite(m1);
        double c0 = 0.0, c1 = 0.0;
        for (int a = 0; a < 4; a++) {
            bad = bad || !isfinite(ph[a]);
            acc[a] += ph[a];
            const double h = ph[a] * ph[a] / S;
            c0 += h * (m0 / (2.0 * kp.A64[a]) + (kp.cE[a][0] + kp.kT64[a][0] * (T - kp.TE)));
            c1 += h * (m1 / (2.0 * kp.A64[a]) + (kp.cE[a][1] + kp.kT64[a][1] * (T - kp.TE)));
        }
        acc[4] += c0;
        acc[5] += c1;
        acc[6] += 1.0 - ph[3];
        acc[7] += bad ? 1.0 : 0.0;
    }
    for (int q = 0; q < 8; q++) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 8; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 8) out[(size_t)k * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// AoS device fields (ring-buffered) <-> FP64 SoA staging for logical planes [k0, k0 + nk).
template <typename R>
__global__ void __launch_bounds__(256) pack_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                  const Ph<R> *__restrict__ phi, const Mu<R> *__restrict__ mu,
                                                  double *__restrict__ phi_soa, double *__restrict__ mu_soa,
                                                  int k0, int nk)
{
    const size_t plane = (size_t)kp.nx * kp.ny, n = plane * nk;
    const int zbase = st->zbase;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(q / plane);
        const size_t c = q % plane;
        const size_t g = plane_off(k0 + kk, kp.nz, zbase, plane) + c;
        if (phi_soa) {
            const Ph<R> p = ldg_ph(phi + g);
            for (int a = 0; a < 4; a++) phi_soa[(size_t)a * n + q] = (double)p.v[a];
        }
        if (mu_soa) {
            const Mu<R> m = ldg_mu(mu + g);
            mu_soa[q] = (double)m.v[0];
            mu_soa[n + q] = (double)m.v[1];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) unpack_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                    Ph<R> *__restrict__ phi, Mu<R> *__restrict__ mu,
                                                    const double *__restrict__ phi_soa,
                                                    const double *__restrict__ mu_soa, int k0, int nk)
{
    const size_t plane = (size_t)kp.nx * kp.ny, n = plane * nk;
    const int zbase = st->zbase;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(q / plane);
        const size_t c = q % plane;
        const size_t g = plane_off(k0 + kk, kp.nz, zbase, plane) + c;
        Ph<R> p;
        for (int a = 0; a < 4; a++) p.v[a] = (R)phi_soa[(size_t)a * n + q];
        st_ph(phi + g, p);
        Mu<R> m;
        m.v[0] = (R)mu_soa[q];
        m.v[1] = (R)mu_soa[n + q];
        st_mu(mu + g, m);
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
constexpr int kTX = 32, kTY = 8;

template <typename R>
static size_t phi_smem_bytes()
{
    constexpr int SN = (kTX + 2) * (kTY + 2), FX = kTY * (kTX + 1), FY = (kTY + 1) * kTX;
    return sizeof(Ph<R>) * (4 * SN + 2 * FX + 2 * FY) + sizeof(Mu<R>) * 4 * kTX * kTY;
}
template <typename R>
static size_t mu_smem_bytes()
{
    constexpr int SN = (kTX + 2) * (kTY + 2), FX = kTY * (kTX + 1), FY = (kTY + 1) * kTX;
    return sizeof(Ph<R>) * 7 * SN + sizeof(Mu<R>) * (3 * SN + 2 * FX + 2 * FY);
}

static inline int grid1d(size_t n, int per_block = 256, int cap = 152 * 32)
{
    size_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

template <typename R>
cudaError_t launch_phi_sweep(const KParams<R> &kp, const Geometry &g, const void *phi, const void *mu,
                             void *phi_out, const DevState *st, const PlaneT<R> *tab, cudaStream_t s)
{
    static bool attr = false;
    const size_t sm = phi_smem_bytes<R>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(phi_sweep_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(g.gx, g.gy, g.gz);
    phi_sweep_kernel<R, kTX, kTY><<<grid, kTX * kTY, sm, s>>>(kp, (const Ph<R> *)phi, (const Mu<R> *)mu,
                                                              (Ph<R> *)phi_out, st, tab);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mu_sweep(const KParams<R> &kp, const Geometry &g, const void *phi_old, const void *phi_new,
                            const void *mu, void *mu_out, const DevState *st, const PlaneT<R> *tab,
                            Partial *parts, cudaStream_t s)
{
    static bool attr = false;
    const size_t sm = mu_smem_bytes<R>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mu_sweep_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(g.gx, g.gy, g.gz);
    mu_sweep_kernel<R, kTX, kTY><<<grid, kTX * kTY, sm, s>>>(kp, (const Ph<R> *)phi_old, (const Ph<R> *)phi_new,
                                                             (const Mu<R> *)mu, (Mu<R> *)mu_out, st, tab, parts);
    return cudaGetLastError();
}

template <typename R>
static size_t fused_smem_bytes()
{
    constexpr int SN = (kTX + 2) * (kTY + 2), SN2 = (kTX + 4) * (kTY + 4);
    constexpr int PFX = (kTX + 3) * (kTY + 2), PFY = (kTX + 2) * (kTY + 3);
    constexpr int FX = kTY * (kTX + 1), FY = (kTY + 1) * kTX;
    return sizeof(Ph<R>) * (3 * SN2 + 3 * SN + PFX + PFY) + sizeof(Mu<R>) * (3 * SN + FX + FY) + 3 * SN2 + 3 * SN;
}

template <typename R>
cudaError_t launch_fused_step(const KParams<R> &kp, const Geometry &g, const void *phi, const void *mu,
                              void *phi_out, void *mu_out, const DevState *st, const PlaneT<R> *tab, Partial *parts,
                              cudaStream_t s)
{
    static bool attr = false;
    const size_t sm = fused_smem_bytes<R>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(g.gx, g.gy, g.gz);
    fused_step_kernel<R, kTX, kTY><<<grid, kTX * kTY, sm, s>>>(kp, (const Ph<R> *)phi, (const Mu<R> *)mu,
                                                               (Ph<R> *)phi_out, (Mu<R> *)mu_out, st, tab, parts);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_finalize(const KParams<R> &kp, DevState *st, const Partial *parts, int nparts, cudaStream_t s)
{
    finalize_kernel<R><<<1, 256, 0, s>>>(kp, st, parts, nparts);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_post(const KParams<R> &kp, const DevState *st, void *phi, void *mu, PlaneT<R> *tab,
                        cudaStream_t s)
{
    // enough threads to fill one full plane per thread-sweep when the window moves
    const size_t work = (size_t)kp.nx * kp.ny;
    post_kernel<R><<<grid1d(work > (size_t)2 * kp.nz ? work : (size_t)2 * kp.nz), 256, 0, s>>>(
        kp, st, (Ph<R> *)phi, (Mu<R> *)mu, tab);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init(const KParams<R> &kp, void *phi, void *mu, const double *seeds, int n_grains, int H,
                        cudaStream_t s)
{
    const size_t n = (size_t)kp.nx * kp.ny * kp.nz;
    init_kernel<R><<<grid1d(n), 256, 0, s>>>(kp, (Ph<R> *)phi, (Mu<R> *)mu, seeds, n_grains, H);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_reduce(const KParams<R> &kp, const DevState *st, const void *phi, const void *mu,
                          double *plane_sums, cudaStream_t s)
{
    reduce_kernel<R><<<kp.nz, 256, 0, s>>>(kp, st, (const Ph<R> *)phi, (const Mu<R> *)mu, plane_sums);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pack(const KParams<R> &kp, const DevState *st, const void *phi, const void *mu, double *phi_soa,
                        double *mu_soa, int k0, int nk, cudaStream_t s)
{
    const size_t n = (size_t)kp.nx * kp.ny * nk;
    pack_kernel<R><<<grid1d(n), 256, 0, s>>>(kp, st, (const Ph<R> *)phi, (const Mu<R> *)mu, phi_soa, mu_soa, k0, nk);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_unpack(const KParams<R> &kp, const DevState *st, void *phi, void *mu, const double *phi_soa,
                          const double *mu_soa, int k0, int nk, cudaStream_t s)
{
    const size_t n = (size_t)kp.nx * kp.ny * nk;
    unpack_kernel<R><<<grid1d(n), 256, 0, s>>>(kp, st, (Ph<R> *)phi, (Mu<R> *)mu, phi_soa, mu_soa, k0, nk);
    return cudaGetLastError();
}

#define PF_INSTANTIATE(R)                                                                                        \
    template cudaError_t launch_phi_sweep<R>(const KParams<R> &, const Geometry &, const void *, const void *,  \
                                             void *, const DevState *, const PlaneT<R> *, cudaStream_t);        \
    template cudaError_t launch_mu_sweep<R>(const KParams<R> &, const Geometry &, const void *, const void *,   \
                                            const void *, void *, const DevState *, const PlaneT<R> *,          \
                                            Partial *, cudaStream_t);                                            \
    template cudaError_t launch_fused_step<R>(const KParams<R> &, const Geometry &, const void *, const void *, \
                                              void *, void *, const DevState *, const PlaneT<R> *, Partial *,     \
                                              cudaStream_t);                                                      \
    template cudaError_t launch_finalize<R>(const KParams<R> &, DevState *, const Partial *, int, cudaStream_t); \
    template cudaError_t launch_post<R>(const KParams<R> &, const DevState *, void *, void *, PlaneT<R> *,       \
                                        cudaStream_t);                                                           \
    template cudaError_t launch_init<R>(const KParams<R> &, void *, void *, const double *, int, int,            \
                                        cudaStream_t);                                                           \
    template cudaError_t launch_reduce<R>(const KParams<R> &, const DevState *, const void *, const void *,      \
                                          double *, cudaStream_t);                                               \
    template cudaError_t launch_pack<R>(const KParams<R> &, const DevState *, const void *, const void *,        \
                                        double *, double *, int, int, cudaStream_t);                             \
    template cudaError_t launch_unpack<R>(const KParams<R> &, const DevState *, void *, void *, const double *,  \
                                          const double *, int, int, cudaStream_t);

}  // namespace pf
