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
template <typename R>
__device__ __forceinline__ bool onehot(const Ph<R> &a)
{
    return a.v[0] == R(1) || a.v[1] == R(1) || a.v[2] == R(1) || a.v[3] == R(1);
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
// staging of one plane-table entry into shared memory (16 words, broadcast afterwards)
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void stage_plane(PlaneT<R> *dst, const PlaneT<R> *src)
{
    if (threadIdx.x < 16) reinterpret_cast<R *>(dst)[threadIdx.x] = __ldg(reinterpret_cast<const R *>(src) + threadIdx.x);
}

// ---------------------------------------------------------------------------------------
// phi-sweep kernel: phi^{n+1} = Proj(phi^n - dt/(tau eps) (rhs - mean rhs))   (Eq. 1, Eq. 2)
// ---------------------------------------------------------------------------------------
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) phi_sweep_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi,
                                                          const Mu<R> *__restrict__ mu,
                                                          Ph<R> *__restrict__ phi_out,
                                                          const DevState *__restrict__ st,
                                                          const PlaneT<R> *__restrict__ tab)
{
    constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ph<R>(*sP)[SX] = reinterpret_cast<Ph<R>(*)[SX]>(smem_raw);
    Ph<R>(*sFx)[TX + 1] = reinterpret_cast<Ph<R>(*)[TX + 1]>(smem_raw + sizeof(Ph<R>) * SX * SY);
    Ph<R>(*sFy)[TX] =
        reinterpret_cast<Ph<R>(*)[TX]>(smem_raw + sizeof(Ph<R>) * (SX * SY + TY * (TX + 1)));
    __shared__ PlaneT<R> sT;

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool valid = i < nx && j < ny;
    const int z0 = blockIdx.z * kp.zchunk;
    const int z1 = min(z0 + kp.zchunk, nz);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;
    const size_t col = (size_t)wrapi(j, ny) * nx + wrapi(i, nx);

    Ph<R> pm = ldg_ph(phi + plane_off(z0 - 1, nz, zbase, plane) + col);
    Ph<R> pc = ldg_ph(phi + plane_off(z0, nz, zbase, plane) + col);
    Ph<R> Fzb = face_phi(kp, pm, pc);

    for (int k = z0; k < z1; ++k) {
        const size_t pk = plane_off(k, nz, zbase, plane);
        Ph<R> pn = ldg_ph(phi + plane_off(k + 1, nz, zbase, plane) + col);
        Mu<R> m = ldg_mu(mu + pk + col);
        __syncthreads();  // readers of the previous plane are done
        stage_plane(&sT, tab + k);
        sP[ty + 1][tx + 1] = pc;
        for (int r = threadIdx.x; r < 2 * (TX + TY); r += NT) {
            int li, lj;
            if (r < TY) {
                li = -1;
                lj = r;
            } else if (r < 2 * TY) {
                li = TX;
                lj = r - TY;
            } else if (r < 2 * TY + TX) {
                li = r - 2 * TY;
                lj = -1;
            } else {
                li = r - 2 * TY - TX;
                lj = TY;
            }
            sP[lj + 1][li + 1] = ldg_ph(phi + pk + (size_t)wrapi(j0 + lj, ny) * nx + wrapi(i0 + li, nx));
        }
        __syncthreads();
        const Ph<R> xm = sP[ty + 1][tx], xp = sP[ty + 1][tx + 2];
        const Ph<R> ym = sP[ty][tx + 1], yp = sP[ty + 2][tx + 1];
        sFx[ty][tx] = face_phi(kp, xm, pc);
        if (tx == TX - 1) sFx[ty][TX] = face_phi(kp, pc, xp);
        sFy[ty][tx] = face_phi(kp, ym, pc);
        if (ty == TY - 1) sFy[TY][tx] = face_phi(kp, pc, yp);
        const Ph<R> Fza = face_phi(kp, pc, pn);
        __syncthreads();
        // bulk cells (one-hot, all six neighbours equal) are fixed points of the step; a warp
        // whose cells are all bulk skips the cell terms (the shortcuts of Section 3.3)
        const bool bulk = onehot(pc) && same(pc, xm) && same(pc, xp) && same(pc, ym) && same(pc, yp) &&
                          same(pc, pm) && same(pc, pn);
        Ph<R> out = pc;
        if (!__all_sync(0xffffffffu, bulk)) {
            out = phi_cell(kp, sT, pc, xm, xp, ym, yp, pm, pn, sFx[ty][tx], sFx[ty][tx + 1], sFy[ty][tx],
                           sFy[ty + 1][tx], Fzb, Fza, m);
        }
        if (valid) st_ph(phi_out + pk + col, out);
        pm = pc;
        pc = pn;
        Fzb = Fza;
    }
}

// ---------------------------------------------------------------------------------------
// mu-sweep pieces (Eq. 3, Eq. 4)
// ---------------------------------------------------------------------------------------

// v = M(phibar) grad mu - J_at on one face.  nL/nR: phi^{n+1} at the two cells, oL/oR:
// phi^n, mL/mR: mu^n.  tan1*/tan2*: phi^{n+1} at the four tangential neighbours of L and R
// for the two tangential directions (the D3C19 stencil): face gradient component
//   (L+e - L-e + R+e - R-e) / (4 dx).
// chatf: chat_a(T_face) for the face temperature.
template <typename R>
__device__ __forceinline__ Mu<R> face_mu(const KParams<R> &kp, const R (&chatf)[4][2], const Ph<R> &nL,
                                         const Ph<R> &nR, const Ph<R> &oL, const Ph<R> &oR, const Mu<R> &mL,
                                         const Mu<R> &mR, const Ph<R> &aLp, const Ph<R> &aLm,
                                         const Ph<R> &aRp, const Ph<R> &aRm, const Ph<R> &bLp,
                                         const Ph<R> &bLm, const Ph<R> &bRp, const Ph<R> &bRm)
{
    R pb[4];
#pragma unroll
    for (int b = 0; b < 4; b++) pb[b] = R(0.5) * (nL.v[b] + nR.v[b]);
    const R S = pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2] + pb[3] * pb[3];
    const R inv_S = R(1) / S;
    R h[4];
#pragma unroll
    for (int b = 0; b < 4; b++) h[b] = pb[b] * pb[b] * inv_S;
    const R M = kp.DinvA[0] * h[0] + kp.DinvA[1] * h[1] + kp.DinvA[2] * h[2] + kp.DinvA[3] * h[3];
    Mu<R> v;
    v.v[0] = M * (mR.v[0] - mL.v[0]) * kp.inv_dx;
    v.v[1] = M * (mR.v[1] - mL.v[1]) * kp.inv_dx;
    // anti-trapping current (Eq. 4, g_a = phi_a); terms skipped per reading R9
    if (pb[3] > R(0) && (pb[0] > R(0) || pb[1] > R(0) || pb[2] > R(0))) {
        // liquid gradient
        R gl[3];
        gl[0] = (nR.v[3] - nL.v[3]) * kp.inv_dx;
        gl[1] = (aLp.v[3] - aLm.v[3] + aRp.v[3] - aRm.v[3]) * kp.inv_4dx;
        gl[2] = (bLp.v[3] - bLm.v[3] + bRp.v[3] - bRm.v[3]) * kp.inv_4dx;
        const R gl2 = gl[0] * gl[0] + gl[1] * gl[1] + gl[2] * gl[2];
        if (gl2 > kp.grad_thr) {
            const R nl = sqrt(gl2);
            const R mb0 = R(0.5) * (mL.v[0] + mR.v[0]);
            const R mb1 = R(0.5) * (mL.v[1] + mR.v[1]);
            const R cl0 = mb0 * kp.inv2A[3] + chatf[3][0];
            const R cl1 = mb1 * kp.inv2A[3] + chatf[3][1];
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
                const R dc0 = cl0 - (mb0 * kp.inv2A[a] + chatf[a][0]);
                const R dc1 = cl1 - (mb1 * kp.inv2A[a] + chatf[a][1]);
                const R nd = ga[0] / na;  // normal component: the face direction is component 0
                v.v[0] = v.v[0] - pref * dc0 * nd;
                v.v[1] = v.v[1] - pref * dc1 * nd;
            }
        }
    }
    return v;
}

// mu update at one cell (Eq. 3, reading R10):
//   mu^{n+1} = mu^n + [dt div v - sum_a c^a(mu^n,T)(h_a(new) - h_a(old)) - sum_a h_a(new) kT_a dT] / chi
template <typename R>
__device__ __forceinline__ Mu<R> mu_cell(const KParams<R> &kp, const PlaneT<R> &pc, const Ph<R> &nP,
                                         const Ph<R> &oP, const Mu<R> &m, R div0, R div1)
{
    R hN[4], hO[4];
    const R iSN = R(1) / (nP.v[0] * nP.v[0] + nP.v[1] * nP.v[1] + nP.v[2] * nP.v[2] + nP.v[3] * nP.v[3]);
    const R iSO = R(1) / (oP.v[0] * oP.v[0] + oP.v[1] * oP.v[1] + oP.v[2] * oP.v[2] + oP.v[3] * oP.v[3]);
#pragma unroll
    for (int a = 0; a < 4; a++) {
        hN[a] = nP.v[a] * nP.v[a] * iSN;
        hO[a] = oP.v[a] * oP.v[a] * iSO;
    }
    R chi = R(0), dphi0 = R(0), dphi1 = R(0), dT0 = R(0), dT1 = R(0);
#pragma unroll
    for (int a = 0; a < 4; a++) {
        chi = chi + hN[a] * kp.inv2A[a];
        const R dh = hN[a] - hO[a];
        dphi0 = dphi0 + (m.v[0] * kp.inv2A[a] + pc.chat[a][0]) * dh;
        dphi1 = dphi1 + (m.v[1] * kp.inv2A[a] + pc.chat[a][1]) * dh;
        dT0 = dT0 + hN[a] * kp.kT[a][0];
        dT1 = dT1 + hN[a] * kp.kT[a][1];
    }
    const R src0 = kp.dt * div0 - dphi0 - dT0 * kp.dTstep;
    const R src1 = kp.dt * div1 - dphi1 - dT1 * kp.dTstep;
    const R ichi = R(1) / chi;
    Mu<R> o;
    o.v[0] = m.v[0] + src0 * ichi;
    o.v[1] = m.v[1] + src1 * ichi;
    return o;
}

template <typename R>
__device__ __forceinline__ bool finite4(const Ph<R> &a)
{
    return isfinite(a.v[0]) && isfinite(a.v[1]) && isfinite(a.v[2]) && isfinite(a.v[3]);
}

// ---------------------------------------------------------------------------------------
// mu-sweep kernel: mu^{n+1} from mu^n, phi^n, phi^{n+1}   (Eq. 3, Eq. 4), with the FP64
// per-CTA partial sums of the window trigger and the non-finite check in its epilogue
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
    constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2, SN = SX * SY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // phi^{n+1}: 3-plane ring (k-1, k, k+1) with a full halo ring incl. corners;
    // phi^n and mu^n: 2-plane ring (k, k+1) with the halo ring.
    Ph<R> *sN = reinterpret_cast<Ph<R> *>(smem_raw);
    Ph<R> *sO = sN + 3 * SN;
    Mu<R> *sM = reinterpret_cast<Mu<R> *>(sO + 2 * SN);
    Mu<R> *sVx = sM + 2 * SN;          // [TY][TX+1]
    Mu<R> *sVy = sVx + TY * (TX + 1);  // [TY+1][TX]
    __shared__ double red[NT / 32][2];
    __shared__ PlaneT<R> sTc, sTf;     // constants of plane k and of the z-face level k+1/2

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int i = i0 + tx, j = j0 + ty;
    const bool valid = i < nx && j < ny;
    const int z0 = blockIdx.z * kp.zchunk;
    const int z1 = min(z0 + kp.zchunk, nz);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;
    const size_t col = (size_t)wrapi(j, ny) * nx + wrapi(i, nx);

    auto load_plane = [&](int k) {
        const size_t pk = plane_off(k, nz, zbase, plane);
        const int sn = ((k % 3) + 3) % 3, s2 = k & 1;
        for (int r = threadIdx.x; r < SN; r += NT) {
            const int li = r % SX - 1, lj = r / SX - 1;
            const size_t g = pk + (size_t)wrapi(j0 + lj, ny) * nx + wrapi(i0 + li, nx);
            sN[sn * SN + r] = ldg_ph(phi_new + g);
            sO[s2 * SN + r] = ldg_ph(phi_old + g);
            sM[s2 * SN + r] = ldg_mu(mu + g);
        }
    };
    auto N = [&](int k, int li, int lj) -> const Ph<R> & {
        return sN[(((k % 3) + 3) % 3) * SN + (lj + 1) * SX + (li + 1)];
    };
    auto O = [&](int k, int li, int lj) -> const Ph<R> & { return sO[(k & 1) * SN + (lj + 1) * SX + (li + 1)]; };
    auto Mm = [&](int k, int li, int lj) -> const Mu<R> & { return sM[(k & 1) * SN + (lj + 1) * SX + (li + 1)]; };

    // z face between logical planes k and k+1 at this thread's column (sTf must hold level k+1/2)
    auto zface = [&](int k) -> Mu<R> {
        Mu<R> v;
        if (k < 0 || k >= nz - 1) {
            v.v[0] = v.v[1] = R(0);  // mirror boundary: zero flux
            return v;
        }
        return face_mu(kp, sTf.chat, N(k, tx, ty), N(k + 1, tx, ty), O(k, tx, ty), O(k + 1, tx, ty),
                       Mm(k, tx, ty), Mm(k + 1, tx, ty), N(k, tx + 1, ty), N(k, tx - 1, ty), N(k + 1, tx + 1, ty),
                       N(k + 1, tx - 1, ty), N(k, tx, ty + 1), N(k, tx, ty - 1), N(k + 1, tx, ty + 1),
                       N(k + 1, tx, ty - 1));
    };

    double liq_def = 0.0;
    bool bad = false;

    load_plane(z0 - 1);
    load_plane(z0);
    if (z0 >= 1) stage_plane(&sTf, tab + nz + (z0 - 1));
    __syncthreads();
    Mu<R> Vzb = zface(z0 - 1);

    for (int k = z0; k < z1; ++k) {
        __syncthreads();  // the previous plane's readers are done before its slots are reused
        load_plane(k + 1);
        stage_plane(&sTc, tab + k);
        if (k < nz - 1) stage_plane(&sTf, tab + nz + k);
        __syncthreads();
        // x face between (tx-1) and tx, and the last one (TX-1, TX)
        {
            const int li = tx - 1;
            sVx[ty * (TX + 1) + tx] =
                face_mu(kp, sTc.chat, N(k, li, ty), N(k, li + 1, ty), O(k, li, ty), O(k, li + 1, ty), Mm(k, li, ty),
                        Mm(k, li + 1, ty), N(k, li, ty + 1), N(k, li, ty - 1), N(k, li + 1, ty + 1),
                        N(k, li + 1, ty - 1), N(k + 1, li, ty), N(k - 1, li, ty), N(k + 1, li + 1, ty),
                        N(k - 1, li + 1, ty));
            if (tx == TX - 1) {
                const int l2 = TX - 1;
                sVx[ty * (TX + 1) + TX] = face_mu(
                    kp, sTc.chat, N(k, l2, ty), N(k, l2 + 1, ty), O(k, l2, ty), O(k, l2 + 1, ty), Mm(k, l2, ty),
                    Mm(k, l2 + 1, ty), N(k, l2, ty + 1), N(k, l2, ty - 1), N(k, l2 + 1, ty + 1),
                    N(k, l2 + 1, ty - 1), N(k + 1, l2, ty), N(k - 1, l2, ty), N(k + 1, l2 + 1, ty),
                    N(k - 1, l2 + 1, ty));
            }
        }
        // y face between (ty-1) and ty, and the last one
        {
            const int lj = ty - 1;
            sVy[ty * TX + tx] =
                face_mu(kp, sTc.chat, N(k, tx, lj), N(k, tx, lj + 1), O(k, tx, lj), O(k, tx, lj + 1), Mm(k, tx, lj),
                        Mm(k, tx, lj + 1), N(k, tx + 1, lj), N(k, tx - 1, lj), N(k, tx + 1, lj + 1),
                        N(k, tx - 1, lj + 1), N(k + 1, tx, lj), N(k - 1, tx, lj), N(k + 1, tx, lj + 1),
                        N(k - 1, tx, lj + 1));
            if (ty == TY - 1) {
                const int l2 = TY - 1;
                sVy[TY * TX + tx] = face_mu(
                    kp, sTc.chat, N(k, tx, l2), N(k, tx, l2 + 1), O(k, tx, l2), O(k, tx, l2 + 1), Mm(k, tx, l2),
                    Mm(k, tx, l2 + 1), N(k, tx + 1, l2), N(k, tx - 1, l2), N(k, tx + 1, l2 + 1),
                    N(k, tx - 1, l2 + 1), N(k + 1, tx, l2), N(k - 1, tx, l2), N(k + 1, tx, l2 + 1),
                    N(k - 1, tx, l2 + 1));
            }
        }
        const Mu<R> Vza = zface(k);
        __syncthreads();
        const Mu<R> vxm = sVx[ty * (TX + 1) + tx], vxp = sVx[ty * (TX + 1) + tx + 1];
        const Mu<R> vym = sVy[ty * TX + tx], vyp = sVy[(ty + 1) * TX + tx];
        R div0 = (vxp.v[0] - vxm.v[0]) * kp.inv_dx;
        R div1 = (vxp.v[1] - vxm.v[1]) * kp.inv_dx;
        div0 = div0 + (vyp.v[0] - vym.v[0]) * kp.inv_dx;
        div1 = div1 + (vyp.v[1] - vym.v[1]) * kp.inv_dx;
        div0 = div0 + (Vza.v[0] - Vzb.v[0]) * kp.inv_dx;
        div1 = div1 + (Vza.v[1] - Vzb.v[1]) * kp.inv_dx;
        const Ph<R> nP = N(k, tx, ty);
        const Mu<R> out = mu_cell(kp, sTc, nP, O(k, tx, ty), Mm(k, tx, ty), div0, div1);
        if (valid) {
            st_mu(mu_out + plane_off(k, nz, zbase, plane) + col, out);
            liq_def += 1.0 - (double)nP.v[3];
            bad = bad || !isfinite(out.v[0]) || !isfinite(out.v[1]) || !finite4(nP);
        }
        Vzb = Vza;
    }

    // FP64 per-CTA partials (fixed order: lanes by a shuffle tree, then warps in order)
    double badv = bad ? 1.0 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        liq_def += __shfl_down_sync(0xffffffffu, liq_def, o);
        badv += __shfl_down_sync(0xffffffffu, badv, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[w][0] = liq_def;
        red[w][1] = badv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
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
    constexpr int SX = kTX + 2, SY = kTY + 2;
    return sizeof(Ph<R>) * (SX * SY + kTY * (kTX + 1) + (kTY + 1) * kTX);
}
template <typename R>
static size_t mu_smem_bytes()
{
    constexpr int SN = (kTX + 2) * (kTY + 2);
    return sizeof(Ph<R>) * 5 * SN + sizeof(Mu<R>) * (2 * SN + kTY * (kTX + 1) + (kTY + 1) * kTX);
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
