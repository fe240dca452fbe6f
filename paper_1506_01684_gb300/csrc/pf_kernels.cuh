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

#include <atomic>
#include <utility>
#include <climits>
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

// Asynchronous global -> shared copies of one cell (cp.async; completion per commit group): the
// sweeps stage the planes ahead straight into their shared-memory ring, with no registers held for
// the copy.  Both addresses are aligned to the cell (16 bytes for a phi cell, 8 or 16 for a mu cell).
__device__ __forceinline__ void cpa16(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(__cvta_generic_to_global(src)) : "memory");
}
__device__ __forceinline__ void cpa8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(__cvta_generic_to_global(src)) : "memory");
}
template <typename T>
__device__ __forceinline__ void cpa_cell(T *dst, const T *src)
{
    static_assert(sizeof(T) % 8 == 0 && sizeof(T) <= 32, "8, 16 or 32-byte cells");
    if constexpr (sizeof(T) == 8) {
        cpa8(dst, src);
    } else {
#pragma unroll
        for (int q = 0; q < (int)sizeof(T) / 16; q++)
            cpa16(reinterpret_cast<char *>(dst) + 16 * q, reinterpret_cast<const char *>(src) + 16 * q);
    }
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Planes of the phi-sweep's shared-memory ring: with asynchronous staging (PF_SWEEP_ASYNC) 8 in FP32
// (7 planes in flight ahead of the plane being updated) and 4 in FP64 (its cells are twice as large);
// without it 4 (one plane ahead, staged through registers).
#ifndef PF_SWEEP_ASYNC
#define PF_SWEEP_ASYNC 0  // 1: 0.7 % faster general planes, 17 % slower whole-domain phi-sweep (GB300)
#endif
template <typename R>
__host__ __device__ constexpr int phi_ring() { return PF_SWEEP_ASYNC ? (sizeof(R) == 4 ? 8 : 4) : 4; }
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

// Programmatic dependent launch (sm_90 and later).  A kernel launched with the programmatic stream
// serialisation attribute may be scheduled before the kernel ahead of it in the stream has finished:
// pdl_wait() blocks until that kernel has completed and its memory operations are visible (it returns
// at once for a launch without the attribute); pdl_trigger() lets the kernel behind this one be
// scheduled once every CTA of this one has triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Liquid map layout: tile-major, the storage planes of one fused-step tile contiguous, so that the
// threads of a warp testing consecutive planes of one tile read consecutive bytes.
__device__ __forceinline__ size_t map_idx(int sp, int tile, int nz) { return (size_t)tile * nz + sp; }

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
    const bool z0 = a.v[0] == z, z1 = a.v[1] == z, z2 = a.v[2] == z, z3 = a.v[3] == z;
    int c = 4;
    c = (a.v[3] == o && z0 && z1 && z2) ? 3 : c;
    c = (a.v[2] == o && z0 && z1 && z3) ? 2 : c;
    c = (a.v[1] == o && z0 && z2 && z3) ? 1 : c;
    c = (a.v[0] == o && z1 && z2 && z3) ? 0 : c;
    return c;
}
template <typename R>
__device__ __forceinline__ bool onehot(const Ph<R> &a)
{
    return code_of(a) < 4;
}
// phase code with a 4-instruction exact test for pure liquid first (bit patterns 0, 0, 0, 1.0f); a
// cell holding -0.0 fails the bit test and gets its code from the full test instead
__device__ __forceinline__ int code_fast(const Ph<float> &a)
{
    const unsigned u0 = __float_as_uint(a.v[0]), u1 = __float_as_uint(a.v[1]), u2 = __float_as_uint(a.v[2]);
    if ((u0 | u1 | u2) == 0u && __float_as_uint(a.v[3]) == 0x3F800000u) return 3;
    return code_of(a);
}
__device__ __forceinline__ int code_fast(const Ph<double> &a)
{
    const unsigned long long u0 = __double_as_longlong(a.v[0]), u1 = __double_as_longlong(a.v[1]),
                             u2 = __double_as_longlong(a.v[2]);
    if ((u0 | u1 | u2) == 0ull && __double_as_longlong(a.v[3]) == 0x3FF0000000000000ll) return 3;
    return code_of(a);
}

// c-th entry of a 4-vector held in kernel parameters, without dynamic indexing
template <typename R>
__device__ __forceinline__ R pick4(const R (&v)[4], int c)
{
    return c == 0 ? v[0] : (c == 1 ? v[1] : (c == 2 ? v[2] : v[3]));
}

// General parabolic thermodynamics (matrix curvatures): a symmetric 2x2 matrix [[s0, s1], [s1, s2]]
template <typename R>
struct Sym2 {
    R s0, s1, s2;
};
// sum_a w_a M_a over the four phases of a table of symmetric matrices
template <typename R>
__device__ __forceinline__ Sym2<R> sym_sum(const R (&M)[4][3], const R *w)
{
    Sym2<R> o;
    o.s0 = M[0][0] * w[0] + M[1][0] * w[1] + M[2][0] * w[2] + M[3][0] * w[3];
    o.s1 = M[0][1] * w[0] + M[1][1] * w[1] + M[2][1] * w[2] + M[3][1] * w[3];
    o.s2 = M[0][2] * w[0] + M[1][2] * w[1] + M[2][2] * w[2] + M[3][2] * w[3];
    return o;
}
// the matrix of phase c (an exactly one-hot cell)
template <typename R>
__device__ __forceinline__ Sym2<R> sym_pick(const R (&M)[4][3], int c)
{
    const R t0[4] = {M[0][0], M[1][0], M[2][0], M[3][0]};
    const R t1[4] = {M[0][1], M[1][1], M[2][1], M[3][1]};
    const R t2[4] = {M[0][2], M[1][2], M[2][2], M[3][2]};
    return Sym2<R>{pick4(t0, c), pick4(t1, c), pick4(t2, c)};
}
// S^{-1} (x0, x1) by the adjugate
template <typename R>
__device__ __forceinline__ void sym_solve(const Sym2<R> &S, R x0, R x1, R &y0, R &y1)
{
    const R idet = R(1) / (S.s0 * S.s2 - S.s1 * S.s1);
    y0 = (S.s2 * x0 - S.s1 * x1) * idet;
    y1 = (S.s0 * x1 - S.s1 * x0) * idet;
}
// SYM (a template flag of the cell functions below): compiled for the symmetric set only (identity
// curvatures, one relaxation time), the general branches left out; the host launches such an
// instantiation only when kp.gen and kp.gen_tau are both 0.
// c^a(mu) = K_a mu + chat_a
template <typename R, bool SYM = false>
__device__ __forceinline__ void c_alpha(const KParams<R> &kp, int a, R m0, R m1, R ch0, R ch1, R &c0, R &c1)
{
    if (!SYM && kp.gen) {
        c0 = kp.K[a][0] * m0 + kp.K[a][1] * m1 + ch0;
        c1 = kp.K[a][1] * m0 + kp.K[a][2] * m1 + ch1;
    } else {
        c0 = m0 * kp.inv2A[a] + ch0;
        c1 = m1 * kp.inv2A[a] + ch1;
    }
}
// dt / (tau(phi) eps) at a cell with phase fractions p (phi^n): the pair-weighted relaxation time,
// tau on a single-phase cell
template <typename R, bool SYM = false>
__device__ __forceinline__ R phi_coef(const KParams<R> &kp, const R *p)
{
    if (SYM || !kp.gen_tau) return kp.c_phi;
    const R w01 = p[0] * p[1], w02 = p[0] * p[2], w03 = p[0] * p[3];
    const R w12 = p[1] * p[2], w13 = p[1] * p[3], w23 = p[2] * p[3];
    const R den = w01 + w02 + w03 + w12 + w13 + w23;
    if (!(den > R(0))) return kp.c_phi;
    const R num = kp.tau_ab[0] * w01 + kp.tau_ab[1] * w02 + kp.tau_ab[2] * w03 + kp.tau_ab[3] * w12 +
                  kp.tau_ab[4] * w13 + kp.tau_ab[5] * w23;
    return kp.dt_eps * den / num;
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

// rhs_a of Eq. 2 at one cell.
//   xm/xp, ym/yp, zm/zp: the six neighbours; F*: the six face terms (minus/plus side).
template <typename R, bool SYM = false>
__device__ __forceinline__ void phi_rhs(const KParams<R> &kp, const PlaneT<R> &pc, const Ph<R> &P, const Ph<R> &xm,
                                        const Ph<R> &xp, const Ph<R> &ym, const Ph<R> &yp, const Ph<R> &zm,
                                        const Ph<R> &zp, const Ph<R> &Fxm, const Ph<R> &Fxp, const Ph<R> &Fym,
                                        const Ph<R> &Fyp, const Ph<R> &Fzm, const Ph<R> &Fzp, const Mu<R> &m,
                                        R (&rhs)[4])
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
        // -(1/2) mu . K_a mu: |mu|^2 / (4 A_a) for the identity form
        const R quad = (!SYM && kp.gen) ? kp.psiK[a][0] * m.v[0] * m.v[0] + kp.psiK[a][1] * m.v[0] * m.v[1] +
                                    kp.psiK[a][2] * m.v[1] * m.v[1]
                              : mu2 * kp.inv4A[a];
        psi[a] = -quad - (m.v[0] * pc.chat[a][0] + m.v[1] * pc.chat[a][1]) + pc.sT[a];
        hpsi = hpsi + p[a] * p[a] * inv_S * psi[a];
    }
#pragma unroll
    for (int a = 0; a < 4; a++) {
        R dps = R(2) * p[a] * (psi[a] - hpsi) * inv_S;
        rhs[a] = pc.epsT * (R(2) * dadp[a] - div[a]) + pc.Toeps * dom[a] + dps;
    }
}

// Full cell update of the phi-sweep at one cell: phi^{n+1} = Proj(phi^n - dt/(tau eps)(rhs - mean rhs)).
template <typename R, bool SYM = false>
__device__ __forceinline__ Ph<R> phi_cell(const KParams<R> &kp, const PlaneT<R> &pc, const Ph<R> &P,
                                          const Ph<R> &xm, const Ph<R> &xp, const Ph<R> &ym,
                                          const Ph<R> &yp, const Ph<R> &zm, const Ph<R> &zp,
                                          const Ph<R> &Fxm, const Ph<R> &Fxp, const Ph<R> &Fym,
                                          const Ph<R> &Fyp, const Ph<R> &Fzm, const Ph<R> &Fzp,
                                          const Mu<R> &m)
{
    R rhs[4];
    phi_rhs<R, SYM>(kp, pc, P, xm, xp, ym, yp, zm, zp, Fxm, Fxp, Fym, Fyp, Fzm, Fzp, m, rhs);
    const R *p = P.v;
    R mean = (rhs[0] + rhs[1] + rhs[2] + rhs[3]) * R(0.25);
    Ph<R> st;
    const R cp = phi_coef<R, SYM>(kp, p);
#pragma unroll
    for (int a = 0; a < 4; a++) st.v[a] = p[a] - cp * (rhs[a] - mean);
    return project_simplex(st);
}

// ---------------------------------------------------------------------------------------
// compensated FP32: a state value is the unevaluated sum hi + lo of two floats; increments
// computed in FP32 from the hi words are accumulated with error-free transformations
// (Knuth's two-sum, Dekker's fast two-sum), so that increments below the FP32 spacing of the
// state are not lost.  The simplex projection then runs in this double-float arithmetic.
// ---------------------------------------------------------------------------------------
struct DF {
    float h, l;
};
__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = a + b;
    return DF{s, b - (s - a)};
}
// The sums renormalise with a full two-sum: after cancellation the low part can exceed the high
// one, where the fast form would leave a pair whose high word is not the rounded value of the pair.
// Every stored pair is canonical (h = fl(h + l)), so its FP64 value splits back into the same two
// words (checkpoints and host reads of the compensated state round-trip exactly).
__device__ __forceinline__ DF df_add_f(DF a, float b)
{
    DF s = two_sum(a.h, b);
    return two_sum(s.h, s.l + a.l);
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.h, b.h);
    return two_sum(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.h, -b.l}); }
__device__ __forceinline__ bool df_pos(DF a) { return a.h > 0.f || (a.h == 0.f && a.l > 0.f); }
__device__ __forceinline__ bool df_less(DF a, DF b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ DF df_scale2(DF a, float p2) { return DF{a.h * p2, a.l * p2}; }  // exact: p2 a power of 2
__device__ __forceinline__ DF df_div3(DF a)
{
    const float q1 = a.h / 3.f;
    const float r = fmaf(-3.f, q1, a.h) + a.l;  // the remainder of a.h is exact in the FMA
    return fast_two_sum(q1, r / 3.f);
}

// Euclidean projection onto the simplex (reading R6) of double-float values.
__device__ __forceinline__ void project_simplex_df(const DF (&u)[4], DF (&o)[4])
{
    DF s[4] = {u[0], u[1], u[2], u[3]};
#define PF_DCS(a, b)                \
    if (df_less(s[a], s[b])) {      \
        const DF t_ = s[a];         \
        s[a] = s[b];                \
        s[b] = t_;                  \
    }
    PF_DCS(0, 1);
    PF_DCS(2, 3);
    PF_DCS(0, 2);
    PF_DCS(1, 3);
    PF_DCS(1, 2);
#undef PF_DCS
    DF theta{0.f, 0.f};
    DF c = s[0];
    DF t = df_add_f(c, -1.f);
    if (df_pos(df_sub(s[0], t))) theta = t;
    c = df_add(c, s[1]);
    t = df_scale2(df_add_f(c, -1.f), 0.5f);
    if (df_pos(df_sub(s[1], t))) theta = t;
    c = df_add(c, s[2]);
    t = df_div3(df_add_f(c, -1.f));
    if (df_pos(df_sub(s[2], t))) theta = t;
    c = df_add(c, s[3]);
    t = df_scale2(df_add_f(c, -1.f), 0.25f);
    if (df_pos(df_sub(s[3], t))) theta = t;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const DF r = df_sub(u[a], theta);
        o[a] = df_pos(r) ? r : DF{0.f, 0.f};
    }
}

// Compensated phi update: the increment -dt/(tau eps)(rhs - mean) is formed in FP32 from the hi
// words and added to hi + lo; the projection runs in double-float.
__device__ __forceinline__ void phi_cell_comp(const KParams<float> &kp, const PlaneT<float> &pc, const Ph<float> &P,
                                              const Ph<float> &Plo, const Ph<float> &xm, const Ph<float> &xp,
                                              const Ph<float> &ym, const Ph<float> &yp, const Ph<float> &zm,
                                              const Ph<float> &zp, const Ph<float> &Fxm, const Ph<float> &Fxp,
                                              const Ph<float> &Fym, const Ph<float> &Fyp, const Ph<float> &Fzm,
                                              const Ph<float> &Fzp, const Mu<float> &m, Ph<float> &out,
                                              Ph<float> &out_lo)
{
    float rhs[4];
    phi_rhs(kp, pc, P, xm, xp, ym, yp, zm, zp, Fxm, Fxp, Fym, Fyp, Fzm, Fzp, m, rhs);
    const float mean = (rhs[0] + rhs[1] + rhs[2] + rhs[3]) * 0.25f;
    DF u[4], o[4];
    const float cp = phi_coef(kp, P.v);
#pragma unroll
    for (int a = 0; a < 4; a++) u[a] = df_add_f(DF{P.v[a], Plo.v[a]}, -(cp * (rhs[a] - mean)));
    project_simplex_df(u, o);
#pragma unroll
    for (int a = 0; a < 4; a++) {
        out.v[a] = o[a].h;
        out_lo.v[a] = o[a].l;
    }
}



// ---------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------
// reciprocal: correctly rounded in both precisions (exact for 1), no full division in FP32
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
// approximate reciprocal (FP32: the hardware's, as the FP32 unit's divisions; FP64: IEEE division), for
// the anti-trapping current only: the mu update's 1/chi and the weights' 1/sum(phi^2) keep the
// correctly rounded one (the compensated state's solute balance depends on them)
__device__ __forceinline__ float rcp_approx(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_approx(double x) { return 1.0 / x; }
// reciprocal square root (the library's, in each precision)
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

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
template <typename R, bool SYM = false>
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
    if (!SYM && kp.gen) {
        // M = sum_a D_a h_a K_a (a 2x2 matrix)
        const Sym2<R> M = sym_sum(kp.DK, h);
        const R d0 = mR.v[0] - mL.v[0], d1 = mR.v[1] - mL.v[1];
        v.v[0] = (M.s0 * d0 + M.s1 * d1) * kp.inv_dx;
        v.v[1] = (M.s1 * d0 + M.s2 * d1) * kp.inv_dx;
    } else {
        const R M = kp.DinvA[0] * h[0] + kp.DinvA[1] * h[1] + kp.DinvA[2] * h[2] + kp.DinvA[3] * h[3];
        const R Mdx = M * kp.inv_dx;  // mobility over the face width, formed once per face
        v.v[0] = Mdx * (mR.v[0] - mL.v[0]);
        v.v[1] = Mdx * (mR.v[1] - mL.v[1]);
    }
    // anti-trapping current (Eq. 4, g_a = phi_a); terms skipped per reading R9
    if (pb[3] > R(0) && (pb[0] > R(0) || pb[1] > R(0) || pb[2] > R(0))) {
        R gl[3];
        gl[0] = (nR.v[3] - nL.v[3]) * kp.inv_dx;
        gl[1] = (aLp.v[3] - aLm.v[3] + aRp.v[3] - aRm.v[3]) * kp.inv_4dx;
        gl[2] = (bLp.v[3] - bLm.v[3] + bRp.v[3] - bRm.v[3]) * kp.inv_4dx;
        const R gl2 = gl[0] * gl[0] + gl[1] * gl[1] + gl[2] * gl[2];
        if (gl2 > kp.grad_thr) {
            const Chat<R> ch = ldg_chat(tf);
#ifndef PF_AT_RSQRT
#define PF_AT_RSQRT 1  // the normals' products from reciprocal square roots (0: square roots and divisions)
#endif
#if PF_AT_RSQRT
            const R inl = rsq(gl2);  // 1 / |grad phi_l|
#else
            const R nl = sqrt(gl2);
#endif
            const R mb0 = R(0.5) * (mL.v[0] + mR.v[0]);
            const R mb1 = R(0.5) * (mL.v[1] + mR.v[1]);
            R cl0, cl1;
            c_alpha<R, SYM>(kp, 3, mb0, mb1, ch.c[3][0], ch.c[3][1], cl0, cl1);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (!(pb[a] > R(0))) continue;
                R ga[3];
                ga[0] = (nR.v[a] - nL.v[a]) * kp.inv_dx;
                ga[1] = (aLp.v[a] - aLm.v[a] + aRp.v[a] - aRm.v[a]) * kp.inv_4dx;
                ga[2] = (bLp.v[a] - bLm.v[a] + bRp.v[a] - bRm.v[a]) * kp.inv_4dx;
                const R ga2 = ga[0] * ga[0] + ga[1] * ga[1] + ga[2] * ga[2];
                if (!(ga2 > kp.grad_thr)) continue;
                const R pdot = R(0.5) * ((nL.v[a] - oL.v[a]) + (nR.v[a] - oR.v[a])) * kp.inv_dt;
#if PF_AT_RSQRT
                // (n_a . n_l) n_a,0 = (g_a . g_l) g_a,0 / (|g_a|^2 |g_l|) and phi_a / sqrt(phi_a phi_l)
                // = phi_a rsqrt(phi_a phi_l): one reciprocal and one reciprocal square root a term
                const R ndn = (ga[0] * gl[0] + ga[1] * gl[1] + ga[2] * gl[2]) * ga[0] * (rcp_approx(ga2) * inl);
                const R pref = kp.at_pref * (pb[a] * rsq(pb[a] * pb[3]) * h[3]) * pdot * ndn;
                R ca0, ca1;
                c_alpha<R, SYM>(kp, a, mb0, mb1, ch.c[a][0], ch.c[a][1], ca0, ca1);
                v.v[0] = v.v[0] - pref * (cl0 - ca0);
                v.v[1] = v.v[1] - pref * (cl1 - ca1);
#else
                const R na = sqrt(ga2);
                const R ndot = (ga[0] * gl[0] + ga[1] * gl[1] + ga[2] * gl[2]) / (na * nl);
                const R pref = kp.at_pref * (pb[a] * h[3] / sqrt(pb[a] * pb[3])) * pdot * ndot;
                R ca0, ca1;
                c_alpha<R, SYM>(kp, a, mb0, mb1, ch.c[a][0], ch.c[a][1], ca0, ca1);
                const R dc0 = cl0 - ca0;
                const R dc1 = cl1 - ca1;
                const R nd = ga[0] / na;  // normal component: the face direction is component 0
                v.v[0] = v.v[0] - pref * dc0 * nd;
                v.v[1] = v.v[1] - pref * dc1 * nd;
#endif
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
template <typename R, bool SYM = false>
__device__ __forceinline__ Mu<R> face_mu(const KParams<R> &kp, const PlaneT<R> *__restrict__ tf, const Ph<R> &nL,
                                         const Ph<R> &nR, const Ph<R> &oL, const Ph<R> &oR, const Mu<R> &mL,
                                         const Mu<R> &mR, const Ph<R> &aLp, const Ph<R> &aLm,
                                         const Ph<R> &aRp, const Ph<R> &aRm, const Ph<R> &bLp,
                                         const Ph<R> &bLm, const Ph<R> &bRp, const Ph<R> &bRm)
{
    if (same(nL, nR) && onehot(nL)) {
        Mu<R> v;
        if (!SYM && kp.gen) {
            const Sym2<R> M = sym_sum(kp.DK, nL.v);
            const R d0 = mR.v[0] - mL.v[0], d1 = mR.v[1] - mL.v[1];
            v.v[0] = (M.s0 * d0 + M.s1 * d1) * kp.inv_dx;
            v.v[1] = (M.s1 * d0 + M.s2 * d1) * kp.inv_dx;
            return v;
        }
        const R M = kp.DinvA[0] * nL.v[0] + kp.DinvA[1] * nL.v[1] + kp.DinvA[2] * nL.v[2] + kp.DinvA[3] * nL.v[3];
        const R Mdx = M * kp.inv_dx;
        v.v[0] = Mdx * (mR.v[0] - mL.v[0]);
        v.v[1] = Mdx * (mR.v[1] - mL.v[1]);
        return v;
    }
    return face_mu_general<R, SYM>(kp, tf, nL, nR, oL, oR, mL, mR, aLp, aLm, aRp, aRm, bLp, bLm, bRp, bRm);
}

// mu update at one cell (Eq. 3, reading R10):
//   mu^{n+1} = mu^n + [dt div v - sum_a c^a(mu^n,T)(h_a(new) - h_a(old)) - sum_a h_a(new) kT_a dT] / chi
// A cell whose phi did not change and is one-hot takes the exact short form (h = phi, no
// phase-change source).
template <typename R, bool SYM = false>
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
            R ca0, ca1;
            c_alpha<R, SYM>(kp, a, m.v[0], m.v[1], ch.c[a][0], ch.c[a][1], ca0, ca1);
            dphi0 = dphi0 + ca0 * dh;
            dphi1 = dphi1 + ca1 * dh;
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
    Mu<R> o;
    if (!SYM && kp.gen) {
        // chi = sum_a h_a K_a (2x2): mu^{n+1} = mu^n + chi^{-1} src
        R i0, i1;
        sym_solve(sym_sum(kp.K, hN), src0, src1, i0, i1);
        o.v[0] = m.v[0] + i0;
        o.v[1] = m.v[1] + i1;
        return o;
    }
    const R ichi = rcp(chi);
    o.v[0] = m.v[0] + src0 * ichi;
    o.v[1] = m.v[1] + src1 * ichi;
    return o;
}

// Compensated mu update: the increment src/chi is formed in FP32 from the hi words (as in mu_cell)
// and accumulated into hi + lo.
__device__ __forceinline__ void mu_cell_comp(const KParams<float> &kp, const PlaneT<float> *__restrict__ tc,
                                             const Ph<float> &nP, const Ph<float> &oP, const Mu<float> &m,
                                             const Mu<float> &mlo, float div0, float div1, Mu<float> &out,
                                             Mu<float> &out_lo)
{
    float hN[4];
    float dphi0 = 0.f, dphi1 = 0.f;
    if (same(nP, oP) && onehot(nP)) {
#pragma unroll
        for (int a = 0; a < 4; a++) hN[a] = nP.v[a];
    } else {
        float hO[4];
        const float iSN = rcp(nP.v[0] * nP.v[0] + nP.v[1] * nP.v[1] + nP.v[2] * nP.v[2] + nP.v[3] * nP.v[3]);
        const float iSO = rcp(oP.v[0] * oP.v[0] + oP.v[1] * oP.v[1] + oP.v[2] * oP.v[2] + oP.v[3] * oP.v[3]);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            hN[a] = nP.v[a] * nP.v[a] * iSN;
            hO[a] = oP.v[a] * oP.v[a] * iSO;
        }
        const Chat<float> ch = ldg_chat(tc);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const float dh = hN[a] - hO[a];
            float ca0, ca1;
            c_alpha(kp, a, m.v[0], m.v[1], ch.c[a][0], ch.c[a][1], ca0, ca1);
            dphi0 = dphi0 + ca0 * dh;
            dphi1 = dphi1 + ca1 * dh;
        }
    }
    float chi = 0.f, dT0 = 0.f, dT1 = 0.f;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        chi = chi + hN[a] * kp.inv2A[a];
        dT0 = dT0 + hN[a] * kp.kT[a][0];
        dT1 = dT1 + hN[a] * kp.kT[a][1];
    }
    const float src0 = kp.dt * div0 - dphi0 - dT0 * kp.dTstep;
    const float src1 = kp.dt * div1 - dphi1 - dT1 * kp.dTstep;
    float i0, i1;
    if (kp.gen) {
        sym_solve(sym_sum(kp.K, hN), src0, src1, i0, i1);
    } else {
        const float ichi = rcp(chi);
        i0 = src0 * ichi;
        i1 = src1 * ichi;
    }
    const DF r0 = df_add_f(DF{m.v[0], mlo.v[0]}, i0);
    const DF r1 = df_add_f(DF{m.v[1], mlo.v[1]}, i1);
    out.v[0] = r0.h;
    out.v[1] = r1.h;
    out_lo.v[0] = r0.l;
    out_lo.v[1] = r1.l;
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
// One CTA's phi-sweep of tile (bx, by), planes [z0, z1).  With tmap_out, also the new field's
// liquid-map entries of those planes (1 when the tile's cells are exactly pure liquid).
template <typename R, int TX, int TY, bool COMP = false, bool SYM = false>
__device__ __forceinline__ void phi_sweep_tile(const KParams<R> &kp, const Ph<R> *__restrict__ phi,
                                               const Mu<R> *__restrict__ mu, Ph<R> *__restrict__ phi_out,
                                               const DevState *__restrict__ st, const PlaneT<R> *__restrict__ tab,
                                               const Ph<R> *__restrict__ phi_lo, Ph<R> *__restrict__ phi_out_lo,
                                               int bx, int by, int z0, int z1, unsigned char *__restrict__ smem_raw,
                                               unsigned char *__restrict__ tmap_out = nullptr,
                                               const unsigned char *__restrict__ tmap_in = nullptr,
                                               int *__restrict__ map_changed = nullptr)
{
    constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2, SN = SX * SY, NR = SN - NT;
    constexpr int FX = TY * (TX + 1), FY = (TY + 1) * TX;
    constexpr int NS = phi_ring<R>(), D = NS - 1;  // ring planes; planes loaded ahead (asynchronous staging)
    static_assert(NR <= NT, "one halo cell per thread at most");
    static_assert((NS & (NS - 1)) == 0 && NS >= 4, "a power-of-two ring of at least 4 planes");
    Ph<R> *sP = reinterpret_cast<Ph<R> *>(smem_raw);  // [NS][SN]
    Ph<R> *sFx = sP + NS * SN;                         // [2][FX]
    Ph<R> *sFy = sFx + 2 * FX;                         // [2][FY]
    Mu<R> *sMu = reinterpret_cast<Mu<R> *>(sFy + 2 * FY);  // [NS][NT]: own-column mu
    Ph<R> *sLo = reinterpret_cast<Ph<R> *>(sMu + NS * NT);  // [NS][NT]: own-column low words (COMP)

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = bx * TX, j0 = by * TY;
    const bool valid = i0 + tx < nx && j0 + ty < ny;
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

#if PF_SWEEP_ASYNC
    // plane k of the ring: copied straight from global memory (one commit group a plane)
    auto issue = [&](int k) {
        const size_t b = plane_off(k, nz, zbase, plane);
        const int sl = k & (NS - 1);
        cpa_cell(sP + sl * SN + s0, phi + b + col0);
        if (s1 >= 0) cpa_cell(sP + sl * SN + s1, phi + b + col1);
        cpa_cell(sMu + sl * NT + tid, mu + b + col0);
        if constexpr (COMP) cpa_cell(sLo + sl * NT + tid, phi_lo + b + col0);
        cpa_commit();
    };
#else
    Ph<R> pf0, pf1, pfl;
    Mu<R> pfm;
    auto prefetch = [&](int k) {
        const size_t b = plane_off(k, nz, zbase, plane);
        pf0 = ldg_ph(phi + b + col0);
        pfm = ldg_mu(mu + b + col0);
        if (s1 >= 0) pf1 = ldg_ph(phi + b + col1);
        if constexpr (COMP) pfl = ldg_ph(phi_lo + b + col0);
    };
    auto commit = [&](int k) {
        Ph<R> *d = sP + (k & 3) * SN;
        d[s0] = pf0;
        if (s1 >= 0) d[s1] = pf1;
        sMu[(k & 3) * NT + tid] = pfm;
        if constexpr (COMP) sLo[(k & 3) * NT + tid] = pfl;
    };
#endif
    auto S = [&](int k, int li, int lj) -> const Ph<R> & { return sP[(k & (NS - 1)) * SN + (lj + 1) * SX + (li + 1)]; };
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

    // prologue: planes z0-1 .. z0+2 in the ring (with asynchronous staging also the planes up to
    // z0+D-1 in flight), faces of plane z0
#if PF_SWEEP_ASYNC
    for (int k = z0 - 1; k <= z0 + D - 1; k++) issue(k);
    cpa_wait<D - 3>();  // planes z0-1 .. z0+2 have landed (this thread's copies)
#else
    for (int k = z0 - 1; k <= z0 + 2; k++) {
        prefetch(k);
        commit(k);
    }
#endif
    __syncthreads();
    Ph<R> pm = S(z0 - 1, tx, ty), pc = S(z0, tx, ty), pn = S(z0 + 1, tx, ty);
    Ph<R> Fz_prev = face_phi(kp, pm, pc), Fz_cur;
    faces(z0, Fz_cur);
#if !PF_SWEEP_ASYNC
    prefetch(z0 + 3);
#endif
    __syncthreads();

    bool out_liquid = true;
    for (int p = z0; p < z1; ++p) {
#if PF_SWEEP_ASYNC
        // plane p+D into the slot of plane p-1 (no thread reads it after the last barrier)
        issue(p + D);
#endif
        // C(p)
        {
            const Ph<R> xm = S(p, tx - 1, ty), xp = S(p, tx + 1, ty);
            const Ph<R> ym = S(p, tx, ty - 1), yp = S(p, tx, ty + 1);
            bool bulk = onehot(pc) && same(pc, xm) && same(pc, xp) && same(pc, ym) && same(pc, yp) &&
                        same(pc, pm) && same(pc, pn);
            Ph<R> out = pc, out_lo;
            if constexpr (COMP) {
                // a compensated bulk cell also needs a zero low word to be a fixed point
                out_lo = sLo[(p & (NS - 1)) * NT + tid];
                bulk = bulk && out_lo.v[0] == R(0) && out_lo.v[1] == R(0) && out_lo.v[2] == R(0) && out_lo.v[3] == R(0);
            }
            // bulk cells (one-hot, all six neighbours equal) are fixed points of the step; a warp
            // whose cells are all bulk skips the cell terms (the shortcuts of Section 3.3)
            if (!__all_sync(0xffffffffu, bulk)) {
                const Ph<R> *fx = sFx + (p & 1) * FX;
                const Ph<R> *fy = sFy + (p & 1) * FY;
                const PlaneT<R> T = ldg_plane(tab + p);
                if constexpr (COMP) {
                    phi_cell_comp(kp, T, pc, out_lo, xm, xp, ym, yp, pm, pn, fx[ty * (TX + 1) + tx],
                                  fx[ty * (TX + 1) + tx + 1], fy[ty * TX + tx], fy[(ty + 1) * TX + tx], Fz_prev, Fz_cur,
                                  sMu[(p & (NS - 1)) * NT + tid], out, out_lo);
                } else {
                    out = phi_cell<R, SYM>(kp, T, pc, xm, xp, ym, yp, pm, pn, fx[ty * (TX + 1) + tx],
                                   fx[ty * (TX + 1) + tx + 1], fy[ty * TX + tx], fy[(ty + 1) * TX + tx], Fz_prev, Fz_cur,
                                   sMu[(p & (NS - 1)) * NT + tid]);
                }
            }
            if (valid) {
                st_ph(phi_out + plane_off(p, nz, zbase, plane) + col0, out);
                if constexpr (COMP) st_ph(phi_out_lo + plane_off(p, nz, zbase, plane) + col0, out_lo);
            }
            out_liquid = !valid || (out.v[3] == R(1) && out.v[0] == R(0) && out.v[1] == R(0) && out.v[2] == R(0));
            if constexpr (COMP)  // exactly pure liquid: zero low words too
                out_liquid = out_liquid && (!valid || (out_lo.v[0] == R(0) && out_lo.v[1] == R(0) &&
                                                       out_lo.v[2] == R(0) && out_lo.v[3] == R(0)));
        }
        // B(p+1), A(p+3)
        Ph<R> Fz_next = Fz_cur;
        Ph<R> pnn = pn;
        if (p + 1 < z1) {
            faces(p + 1, Fz_next);
            pnn = S(p + 2, tx, ty);
        }
#if PF_SWEEP_ASYNC
        cpa_wait<D - 3>();  // plane p+3 has landed: the next iteration's faces read it
#else
        commit(p + 3);
        prefetch(p + 4);
#endif
        if (tmap_out) {
            // the barrier also gives the map entry of the new plane p
            const int all = __syncthreads_and(out_liquid);
            if (tid == 0) {
                const size_t mi = map_idx((int)(plane_off(p, nz, zbase, plane) / plane), by * kp.tgx + bx, nz);
                tmap_out[mi] = all ? 1 : 0;
                // a tile plane whose pure-liquid status changed invalidates the step's plan
                if (map_changed && tmap_in[mi] != (all ? 1 : 0)) atomicOr(map_changed, 1);
            }
        } else {
            __syncthreads();
        }
        pm = pc;
        pc = pn;
        pn = pnn;
        Fz_prev = Fz_cur;
        Fz_cur = Fz_next;
    }
#if PF_SWEEP_ASYNC
    cpa_wait<0>();  // no copy of this tile lands in shared memory after the tile is done
#endif
}

template <typename R, int TX, int TY, bool COMP = false>
__global__ void __launch_bounds__(TX *TY) phi_sweep_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi,
                                                          const Mu<R> *__restrict__ mu,
                                                          Ph<R> *__restrict__ phi_out,
                                                          const DevState *__restrict__ st,
                                                          const PlaneT<R> *__restrict__ tab,
                                                          const Ph<R> *__restrict__ phi_lo = nullptr,
                                                          Ph<R> *__restrict__ phi_out_lo = nullptr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int z0 = blockIdx.z * kp.zchunk;
    phi_sweep_tile<R, TX, TY, COMP>(kp, phi, mu, phi_out, st, tab, phi_lo, phi_out_lo, blockIdx.x, blockIdx.y, z0,
                                    min(z0 + kp.zchunk, kp.nz), smem_raw);
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
// One CTA's mu-sweep of tile (bx, by), planes [z0, z1); its FP64 partial sums go to *part, with
// `words` words a cell as its algorithmic bytes.  With splits (the step's plan), phi^{n+1} of a
// tile plane that the lean kernel updates is e_l by construction and is taken as such instead of
// being read (the lean kernel may still be writing it).
template <typename R, int TX, int TY, bool COMP = false, bool SYM = false>
__device__ __forceinline__ void mu_sweep_tile(const KParams<R> &kp, const Ph<R> *__restrict__ phi_old,
                                              const Ph<R> *__restrict__ phi_new, const Mu<R> *__restrict__ mu,
                                              Mu<R> *__restrict__ mu_out, const DevState *__restrict__ st,
                                              const PlaneT<R> *__restrict__ tab, Partial *__restrict__ part,
                                              const Mu<R> *__restrict__ mu_lo, Mu<R> *__restrict__ mu_out_lo, int bx,
                                              int by, int z0, int z1, unsigned char *__restrict__ smem_raw,
                                              double words, const int2 *__restrict__ splits = nullptr,
                                              int split_zchunk = 1)
{
    constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2, SN = SX * SY, NR = SN - NT;
    constexpr int FX = TY * (TX + 1), FY = (TY + 1) * TX;
    static_assert(NR <= NT, "one halo cell per thread at most");
    Ph<R> *sN = reinterpret_cast<Ph<R> *>(smem_raw);  // [4][SN] phi^{n+1}
    Ph<R> *sO = sN + 4 * SN;                           // [3][SN] phi^n
    Mu<R> *sM = reinterpret_cast<Mu<R> *>(sO + 3 * SN);  // [3][SN] mu^n
    Mu<R> *sVx = sM + 3 * SN;                          // [2][FX]
    Mu<R> *sVy = sVx + 2 * FX;                         // [2][FY]
    __shared__ double red[NT / 32][2];

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = bx * TX, j0 = by * TY;
    const bool valid = i0 + tx < nx && j0 + ty < ny;
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;

    const int s0 = (ty + 1) * SX + (tx + 1);
    const int col0 = wrapi(j0 + ty, ny) * nx + wrapi(i0 + tx, nx);
    int s1 = -1, col1 = 0, tile1 = 0;
    if (tid < NR) {
        int li, lj;
        ring_cell<TX, TY>(tid, li, lj);
        s1 = (lj + 1) * SX + (li + 1);
        const int wi = wrapi(i0 + li, nx), wj = wrapi(j0 + lj, ny);
        col1 = wj * nx + wi;
        tile1 = (wj / TY) * kp.tgx + wi / TX;  // the ring cell's tile in the plan's grid
    }
    const int tile0 = by * kp.tgx + bx;
    const int ntl = kp.tgx * kp.tgy;
    const bool xtra_y = ty == 0;
    const bool xtra_x = ty == 1 % TY && tx < TY;
    const bool counted = kp.gny == 0 || (j0 + ty >= kp.red_j0 && j0 + ty < kp.red_j1);

    Ph<R> pfN0, pfN1, pfO0, pfO1;
    Mu<R> pfM0, pfM1;
    auto mod3 = [](int k) { return (k + 3) % 3; };  // k >= -3
    // Whether the prefetched plane of this thread's own and ring cell is a lean plane of the step's
    // plan (phi^{n+1} = e_l by construction there: not read, substituted when stored to shared
    // memory).  The splits of the two tiles are kept for the current z chunk, so that no global load
    // sits between a prefetch and the compute it is meant to overlap.
    bool leanN0 = false, leanN1 = false;
    int sp_chunk = -1;
    int2 sp0 = make_int2(0, 0), sp1 = make_int2(0, 0);
    auto prefetch = [&](int k) {
        const size_t b = plane_off(k, nz, zbase, plane);
        if (splits) {
            const int kc = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
            const int ch = kc / split_zchunk;  // the same for every thread of the CTA
            if (ch != sp_chunk) {
                sp_chunk = ch;
                sp0 = splits[ch * ntl + tile0];
                if (s1 >= 0) sp1 = splits[ch * ntl + tile1];
            }
            leanN0 = kc < sp0.x || kc >= sp0.y;
            leanN1 = s1 >= 0 && (kc < sp1.x || kc >= sp1.y);
        }
        if (!leanN0) pfN0 = ldg_ph(phi_new + b + col0);
        pfO0 = ldg_ph(phi_old + b + col0);
        pfM0 = ldg_mu(mu + b + col0);
        if (s1 >= 0) {
            if (!leanN1) pfN1 = ldg_ph(phi_new + b + col1);
            pfO1 = ldg_ph(phi_old + b + col1);
            pfM1 = ldg_mu(mu + b + col1);
        }
    };
    auto commitN = [&](int k) {
        Ph<R> liq;
        liq.v[0] = liq.v[1] = liq.v[2] = R(0);
        liq.v[3] = R(1);
        Ph<R> *d = sN + (k & 3) * SN;
        d[s0] = leanN0 ? liq : pfN0;
        if (s1 >= 0) d[s1] = leanN1 ? liq : pfN1;
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
        return face_mu<R, SYM>(kp, tab + q, N(q, li, lj), N(q, li + 1, lj), O(q, li, lj), O(q, li + 1, lj), Mm(q, li, lj),
                       Mm(q, li + 1, lj), N(q, li, lj + 1), N(q, li, lj - 1), N(q, li + 1, lj + 1),
                       N(q, li + 1, lj - 1), N(q + 1, li, lj), N(q - 1, li, lj), N(q + 1, li + 1, lj),
                       N(q - 1, li + 1, lj));
    };
    auto yface = [&](int q, int li, int lj) -> Mu<R> {
        return face_mu<R, SYM>(kp, tab + q, N(q, li, lj), N(q, li, lj + 1), O(q, li, lj), O(q, li, lj + 1), Mm(q, li, lj),
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
        return face_mu<R, SYM>(kp, tab + nz + q, N(q, tx, ty), N(q + 1, tx, ty), O(q, tx, ty), O(q + 1, tx, ty),
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
            Mu<R> out;
            if constexpr (COMP) {
                const Mu<R> mlo = ldg_mu(mu_lo + plane_off(p, nz, zbase, plane) + col0);
                Mu<R> out_lo;
                mu_cell_comp(kp, tab + p, ownN, ownO, ownM, mlo, div0, div1, out, out_lo);
                if (valid) st_mu(mu_out_lo + plane_off(p, nz, zbase, plane) + col0, out_lo);
            } else {
                out = mu_cell<R, SYM>(kp, tab + p, ownN, ownO, ownM, div0, div1);
            }
            if (valid) {
                st_mu(mu_out + plane_off(p, nz, zbase, plane) + col0, out);
                if (counted) {  // (a slab's ghost rows are not its own)
                    liq_def += 1.0 - (double)ownN.v[3];
                    bad = bad || !isfinite(out.v[0]) || !isfinite(out.v[1]) || !finite4(ownN);
                }
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
        part->liq_deficit = a;
        part->nonfinite = b;
        const double cells = (double)max(0, min(TX, nx - i0)) * (double)max(0, min(TY, ny - j0)) * (double)(z1 - z0);
        part->bytes = cells * (double)sizeof(R) * words;
        part->timeout = 0.0;
    }
}

template <typename R, int TX, int TY, bool COMP = false>
__global__ void __launch_bounds__(TX *TY) mu_sweep_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi_old,
                                                         const Ph<R> *__restrict__ phi_new,
                                                         const Mu<R> *__restrict__ mu,
                                                         Mu<R> *__restrict__ mu_out,
                                                         const DevState *__restrict__ st,
                                                         const PlaneT<R> *__restrict__ tab,
                                                         Partial *__restrict__ partials,
                                                         const Mu<R> *__restrict__ mu_lo = nullptr,
                                                         Mu<R> *__restrict__ mu_out_lo = nullptr)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int z0 = blockIdx.z * kp.zchunk;
    // this sweep: phi^n, phi^{n+1}, mu^n in, mu^{n+1} out (12 words a cell); the compensated state
    // adds the low words of mu in and out
    mu_sweep_tile<R, TX, TY, COMP>(kp, phi_old, phi_new, mu, mu_out, st, tab, partials + bid, mu_lo, mu_out_lo,
                                   blockIdx.x, blockIdx.y, z0, min(z0 + kp.zchunk, kp.nz), smem_raw,
                                   COMP ? 16.0 : 12.0);
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
        if (kp.gen) {
            const Sym2<R> M = sym_pick(kp.DK, cL);
            const R d0 = mR.v[0] - mL.v[0], d1 = mR.v[1] - mL.v[1];
            v.v[0] = (M.s0 * d0 + M.s1 * d1) * kp.inv_dx;
            v.v[1] = (M.s1 * d0 + M.s2 * d1) * kp.inv_dx;
            return v;
        }
        const R M = pick4(kp.DinvA, cL);
        const R Mdx = M * kp.inv_dx;
        v.v[0] = Mdx * (mR.v[0] - mL.v[0]);
        v.v[1] = Mdx * (mR.v[1] - mL.v[1]);
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
        Mu<R> o;
        if (kp.gen) {
            R i0, i1;
            sym_solve(sym_pick(kp.K, cN), src0, src1, i0, i1);
            o.v[0] = m.v[0] + i0;
            o.v[1] = m.v[1] + i1;
            return o;
        }
        const R ichi = rcp(chi);
        o.v[0] = m.v[0] + src0 * ichi;
        o.v[1] = m.v[1] + src1 * ichi;
        return o;
    }
    return mu_cell(kp, tc, nP, oP, m, div0, div1);
}

// Fluxes and mu^{n+1} of a pure-liquid cell whose neighbourhood is pure liquid in phi^n and
// phi^{n+1}: constant mobility, no anti-trapping current, h = phi -- the short forms of
// face_mu_coded and mu_cell_coded for equal codes, kept in one place so that every path that
// takes them evaluates the same expressions.
template <typename R>
__device__ __forceinline__ Mu<R> quiet_flux(const KParams<R> &kp, const Mu<R> &a, const Mu<R> &b)
{
    // flux of the face from cell a to cell b
    Mu<R> v;
    if (kp.gen) {
        const R d0 = b.v[0] - a.v[0], d1 = b.v[1] - a.v[1];
        v.v[0] = (kp.DK[3][0] * d0 + kp.DK[3][1] * d1) * kp.inv_dx;
        v.v[1] = (kp.DK[3][1] * d0 + kp.DK[3][2] * d1) * kp.inv_dx;
        return v;
    }
    const R Mdx = kp.DinvA[3] * kp.inv_dx;
    v.v[0] = Mdx * (b.v[0] - a.v[0]);
    v.v[1] = Mdx * (b.v[1] - a.v[1]);
    return v;
}
template <typename R>
__device__ __forceinline__ Mu<R> quiet_zflux(const KParams<R> &kp, const Mu<R> &a, const Mu<R> &b)
{
    return quiet_flux(kp, a, b);
}
// mu^{n+1} of a pure-liquid cell from its six face fluxes
template <typename R>
__device__ __forceinline__ Mu<R> quiet_mu_update(const KParams<R> &kp, const Mu<R> &mP, const Mu<R> &vxm,
                                                 const Mu<R> &vxp, const Mu<R> &vym, const Mu<R> &vyp,
                                                 const Mu<R> &Vz_lo, const Mu<R> &Vz_hi)
{
    R div0 = (vxp.v[0] - vxm.v[0]) * kp.inv_dx;
    R div1 = (vxp.v[1] - vxm.v[1]) * kp.inv_dx;
    div0 = div0 + (vyp.v[0] - vym.v[0]) * kp.inv_dx;
    div1 = div1 + (vyp.v[1] - vym.v[1]) * kp.inv_dx;
    div0 = div0 + (Vz_hi.v[0] - Vz_lo.v[0]) * kp.inv_dx;
    div1 = div1 + (Vz_hi.v[1] - Vz_lo.v[1]) * kp.inv_dx;
    Ph<R> liquid;
    liquid.v[0] = liquid.v[1] = liquid.v[2] = R(0);
    liquid.v[3] = R(1);
    return mu_cell_coded(kp, (const PlaneT<R> *)nullptr, 3, 3, liquid, liquid, mP, div0, div1);
}
template <typename R>
__device__ __forceinline__ Mu<R> quiet_mu_cell(const KParams<R> &kp, const PlaneT<R> *__restrict__ tc, const Mu<R> &mP,
                                               const Mu<R> &mxm, const Mu<R> &mxp, const Mu<R> &mym,
                                               const Mu<R> &myp, const Mu<R> &Vz_lo, const Mu<R> &Vz_hi)
{
    (void)tc;  // a liquid cell needs no temperature-dependent constant
    return quiet_mu_update(kp, mP, quiet_flux(kp, mxm, mP), quiet_flux(kp, mP, mxp), quiet_flux(kp, mym, mP),
                           quiet_flux(kp, mP, myp), Vz_lo, Vz_hi);
}

// Lean / general split of the z chunk [z0, z1) of tile (bx, by).  Plane q is lean when phi^n is
// pure liquid (liquid map of the source field) on the tile's 2-ring region over the planes
// q-2 .. q+2: then phi^{n+1}(q) = phi^n(q) = e_l and every mu face of the plane takes the quiet
// form (constant mobility, no anti-trapping current).  With kmin / kmax the lowest / highest plane
// of z0-2 .. z1+1 that is not pure liquid, the lean planes are [z0, lo_end) and [hi_beg, z1); the
// general path runs on [lo_end, hi_beg).  CTA-wide: every one of the NTH threads calls it (one
// barrier); kred is NTH/32 pairs of shared ints.
// The fused-step tiles that hold tile (bx, by)'s 2-ring region: its own, and those of the columns
// i0-2, i0-1, i0+w, i0+w+1 (rows alike; with a narrow last tile these can lie two tiles away).
// u* flags mark the first occurrence of each distinct tile.
template <int TX, int TY>
struct RingTiles {
    int xs[5], ys[5];
    bool ux[5], uy[5];
    __device__ __forceinline__ RingTiles(int nx, int ny, int bx, int by)
    {
        const int i0 = bx * TX, j0 = by * TY;
        const int w = min(TX, nx - i0), hgt = min(TY, ny - j0);
        xs[0] = bx;
        xs[1] = wrapi(i0 - 2, nx) / TX;
        xs[2] = wrapi(i0 - 1, nx) / TX;
        xs[3] = wrapi(i0 + w, nx) / TX;
        xs[4] = wrapi(i0 + w + 1, nx) / TX;
        ys[0] = by;
        ys[1] = wrapi(j0 - 2, ny) / TY;
        ys[2] = wrapi(j0 - 1, ny) / TY;
        ys[3] = wrapi(j0 + hgt, ny) / TY;
        ys[4] = wrapi(j0 + hgt + 1, ny) / TY;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            bool ux_ = true, uy_ = true;
#pragma unroll
            for (int d = 0; d < c; d++) {
                ux_ = ux_ && xs[d] != xs[c];
                uy_ = uy_ && ys[d] != ys[c];
            }
            ux[c] = ux_;
            uy[c] = uy_;
        }
    }
    // whether every cell of the 2-ring region is pure liquid in logical plane k (clamped to the
    // domain: the zero-gradient mirror) according to the liquid map
    __device__ __forceinline__ bool liquid(const unsigned char *__restrict__ tmap, int tgx, int ntl, int nz, int zbase,
                                           int k) const
    {
        const int kc = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
        const int sp = kc + zbase >= nz ? kc + zbase - nz : kc + zbase;
        (void)ntl;
        bool ok = true;
#pragma unroll
        for (int r = 0; r < 5; r++)
#pragma unroll
            for (int c = 0; c < 5; c++)
                if (uy[r] && ux[c]) ok = ok & (tmap[map_idx(sp, ys[r] * tgx + xs[c], nz)] == 1);
        return ok;
    }
};

// Lean / general split of the z chunk [z0, z1) of tile (bx, by).  Plane q is lean when phi^n is
// pure liquid (liquid map of the source field) on the tile's 2-ring region over the planes
// q-2 .. q+2: then phi^{n+1}(q) = phi^n(q) = e_l and every mu face of the plane takes the quiet
// form (constant mobility, no anti-trapping current).  With kmin / kmax the lowest / highest plane
// of z0-2 .. z1+1 that is not pure liquid, the lean planes are [z0, lo_end) and [hi_beg, z1); the
// general path runs on [lo_end, hi_beg).
__device__ __forceinline__ void split_from(int z0, int z1, int kmin, int kmax, int &lo_end, int &hi_beg)
{
    lo_end = kmin == INT_MAX ? z1 : max(z0, min(z1, kmin - 2));
    hi_beg = kmin == INT_MAX ? z1 : min(z1, max(lo_end, kmax + 3));
}
// CTA-wide (all NTH threads call it; one barrier); kred is NTH/32 pairs of shared ints.
template <int TX, int TY, int NTH>
__device__ __forceinline__ void lean_split(const unsigned char *__restrict__ tmap_in, int tgx, int tgy, int nx, int ny,
                                           int nz, int zbase, int bx, int by, int z0, int z1, int (*kred)[2],
                                           int &lo_end, int &hi_beg)
{
    const int tid = threadIdx.x;
    const RingTiles<TX, TY> rt(nx, ny, bx, by);
    int kmin = INT_MAX, kmax = INT_MIN;
    for (int k = z0 - 2 + tid; k < z1 + 2; k += NTH)
        if (!rt.liquid(tmap_in, tgx, tgx * tgy, nz, zbase, k)) {
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if ((tid & 31) == 0) {
        kred[tid >> 5][0] = kmin;
        kred[tid >> 5][1] = kmax;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NTH / 32; q++) {
        kmin = min(kmin, kred[q][0]);
        kmax = max(kmax, kred[q][1]);
    }
    split_from(z0, z1, kmin, kmax, lo_end, hi_beg);
}

// Plan of a fused step with the lean kernel: 64 threads (group sub of the 256-thread CTA) compute
// the split of the (tile, z chunk) item `item` (item = bz * tiles + tile, the fused grid's CTA
// order).  A thread tests up to PER planes of the chunk and its 2-plane margins (zchunk + 4 <= 64
// PER), with all their map loads issued before the first test.  Every thread of the CTA calls it
// (one barrier); kred is 8 pairs of shared ints.
template <int TX, int TY, int PER>
__device__ __forceinline__ void plan_item(int nx, int ny, int nz, int tgx, int tgy, int zchunk, int zbase,
                                          const unsigned char *__restrict__ tmap_in, int item, bool live,
                                          int (*kred)[2], int &lo_end, int &hi_beg)
{
    const int ntl = tgx * tgy;
    const int sub = threadIdx.x >> 6, t64 = threadIdx.x & 63, w = threadIdx.x >> 5;
    int kmin = INT_MAX, kmax = INT_MIN;
    int z0 = 0, z1 = 0;
    if (live) {
        const int bz = item / ntl, tile = item % ntl;
        z0 = bz * zchunk;
        z1 = min(z0 + zchunk, nz);
        const RingTiles<TX, TY> rt(nx, ny, tile % tgx, tile / tgx);
        bool liq[PER];
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int k = z0 - 2 + t64 + 64 * r;
            liq[r] = k >= z1 + 2 || rt.liquid(tmap_in, tgx, ntl, nz, zbase, k);
        }
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int k = z0 - 2 + t64 + 64 * r;
            if (!liq[r]) {
                kmin = min(kmin, k);
                kmax = max(kmax, k);
            }
        }
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if ((threadIdx.x & 31) == 0) {
        kred[w][0] = kmin;
        kred[w][1] = kmax;
    }
    __syncthreads();
    kmin = min(kred[2 * sub][0], kred[2 * sub + 1][0]);
    kmax = max(kred[2 * sub][1], kred[2 * sub + 1][1]);
    split_from(z0, z1, kmin, kmax, lo_end, hi_beg);
}
__device__ __forceinline__ void zero_partial(Partial *p)
{
    Partial z;
    z.liq_deficit = z.nonfinite = z.bytes = z.timeout = 0.0;
    *p = z;
}

// Work units of the general planes.  With G items on the list and `slots` persistent CTAs, each item's
// general range [lo, hi) is cut into U = max(1, min(kMaxUnits, slots / G)) units of nearly equal length
// (unit u: lo + len u / U .. lo + len (u + 1) / U; a unit may be empty), so that a short list still gives
// every CTA a unit: a z-marching unit pays a prologue, so items are cut only when CTAs would idle.
__device__ __forceinline__ int general_units(unsigned G, int slots)
{
    const int u = G > 0u ? slots / (int)G : 1;
    return u < 1 ? 1 : (u > kMaxUnits ? kMaxUnits : u);
}
__device__ __forceinline__ void unit_range(int lo, int hi, int U, int u, int &a, int &b)
{
    const int len = hi - lo;
    a = lo + (len * u) / U;
    b = lo + (len * (u + 1)) / U;
}

// Plan of one domain: four items per CTA; items with general planes are appended to glist (count
// in stats->gcount) for the general-plane kernels, the partials of the others are zeroed (their
// planes are all lean: no liquid deficit, no general-path value).
constexpr int PLAN_PER = 5;
template <int TX, int TY>
__global__ void __launch_bounds__(256) plan_kernel(int nx, int ny, int nz, int tgx, int tgy, int zchunk, int gz,
                                                   const DevState *__restrict__ st,
                                                   const unsigned char *__restrict__ tmap_in, int2 *__restrict__ splits,
                                                   int *__restrict__ glist, LeanStats *__restrict__ stats,
                                                   Partial *__restrict__ parts)
{
    __shared__ int kred[8][2];
    pdl_wait();  // the previous step's post kernel (window fill, map entries, zbase)
    pdl_trigger();
    // No liquid-map entry changed and the window did not move since the last plan: its splits, list
    // and zeroed partials still hold (finalize keeps the list then)
#ifndef PF_PLAN_REUSE
#define PF_PLAN_REUSE 1
#endif
    if (PF_PLAN_REUSE && *(volatile int *)&stats->plan_valid) return;
    const int item = blockIdx.x * 4 + (threadIdx.x >> 6);
    const bool live = item < tgx * tgy * gz;
    int lo_end, hi_beg;
    plan_item<TX, TY, PLAN_PER>(nx, ny, nz, tgx, tgy, zchunk, st->zbase, tmap_in, item, live, kred, lo_end, hi_beg);
    if (live && (threadIdx.x & 63) == 0) {
        splits[item] = make_int2(lo_end, hi_beg);
        if (hi_beg > lo_end)
            glist[atomicAdd(&stats->gcount, 1u)] = item;
        else
            zero_partial(parts + item);
    }
}

// One CTA's work of the fused step: tile (bx, by) of x-y columns, z chunk bz.  Shared by the
// single-domain kernel (tile = block index) and the batched persistent kernel (tile = work item).
template <typename R, int TX, int TY>
__device__ __forceinline__ void fused_tile(const KParams<R> &kp, const Ph<R> *__restrict__ phi,
                                           const Mu<R> *__restrict__ mu, Ph<R> *__restrict__ phi_out,
                                           Mu<R> *__restrict__ mu_out, const DevState *__restrict__ st,
                                           const PlaneT<R> *__restrict__ tab, Partial *__restrict__ part, int bx,
                                           int by, int bz, unsigned char *__restrict__ smem_raw,
                                           const unsigned char *__restrict__ tmap_in,
                                           unsigned char *__restrict__ tmap_out, bool lean_here = true,
                                           const int2 *__restrict__ split = nullptr)
{
    constexpr int NT = TX * TY;
    constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY, NR = SN - NT;  // tile + 1-ring
    constexpr int SX2 = TX + 4, SY2 = TY + 4, SN2 = SX2 * SY2;           // tile + 2-ring
    constexpr int PFX = (TX + 3) * (TY + 2), PFY = (TX + 2) * (TY + 3);   // phi faces of the 1-ring region
    constexpr int FX = TY * (TX + 1), FY = (TY + 1) * TX;                 // mu faces of the tile
    static_assert(NR <= NT && SN2 <= 2 * NT, "tile too small for the slot layout");
    // 4-plane rings: the commit of plane q+3 lands in the slot of plane q-1, which no thread
    // reads once the barrier of plane q has passed (quiet planes have no later barrier)
    Ph<R> *sO = reinterpret_cast<Ph<R> *>(smem_raw);  // [4][SN2] phi^n
    Ph<R> *sN = sO + 4 * SN2;                           // [4][SN]  phi^{n+1}
    Ph<R> *sF = sN + 4 * SN;                            // [PFX + PFY] phi faces (x, then y)
    Mu<R> *sM = reinterpret_cast<Mu<R> *>(sF + PFX + PFY);  // [4][SN] mu^n
    Mu<R> *sVx = sM + 4 * SN;                           // [FX]
    Mu<R> *sVy = sVx + FX;                              // [FY]
    Ph<R> *sFz = reinterpret_cast<Ph<R> *>(sVy + FY);  // [2][SN] phi z-face terms of the 1-ring cells
    unsigned char *cO = reinterpret_cast<unsigned char *>(sFz + 2 * SN);  // [4][SN2]
    unsigned char *cN = cO + 4 * SN2;                                      // [4][SN]
    __shared__ double red[NT / 32][2];
    __shared__ int kred[NT / 32][2];

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int i0 = bx * TX, j0 = by * TY;
    const bool valid = i0 + tx < nx && j0 + ty < ny;
    int z0 = bz * kp.zchunk;  // narrowed to the planes of the general path below
    int z1 = min(z0 + kp.zchunk, nz);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;
    const int col_own = wrapi(j0 + ty, ny) * nx + wrapi(i0 + tx, nx);
    const int t1 = (ty + 1) * SX + (tx + 1);   // own cell, 1-ring layout
    const int t2 = (ty + 2) * SX2 + (tx + 2);  // own cell, 2-ring layout
    const int ntl = kp.tgx * kp.tgy, tile = by * kp.tgx + bx;
    auto splane = [&](int k) {  // storage plane of logical plane k (zero-gradient mirror first)
        const int kc = k < 0 ? 0 : (k >= nz ? nz - 1 : k);
        const int sp = kc + zbase;
        return sp >= nz ? sp - nz : sp;
    };

    // FP64 per-CTA partials (fixed order: lanes by a shuffle tree, then warps in order)
    auto epilogue = [&](double liq_def, bool bad, double bytes) {
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
            part->liq_deficit = a;
            part->nonfinite = b;
            part->bytes = bytes;
            part->timeout = 0.0;
        }
    };
    // the tile's cells per plane (a ragged tile at the domain edge holds fewer)
    const double tile_cells = (double)min(TX, nx - i0) * (double)min(TY, ny - j0);
    double lean_bytes = 0.0;

    // ---- lean segments (see lean_split): they need no shared memory and no barrier.  With
    // lean_here = false they belong to lean_step_kernel, launched beside this one, and this CTA
    // runs only the general planes between them (split: the chunk's split, precomputed by
    // plan_kernel).
    bool bad = false;
    if (tmap_in) {
        int lo_end, hi_beg;
        if (split) {
            lo_end = split->x;
            hi_beg = split->y;
        } else {
            lean_split<TX, TY, NT>(tmap_in, kp.tgx, kp.tgy, nx, ny, nz, zbase, bx, by, z0, z1, kred, lo_end, hi_beg);
        }
        const int i = i0 + tx, j = j0 + ty;
        const int cxm = wrapi(j, ny) * nx + wrapi(i - 1, nx), cxp = wrapi(j, ny) * nx + wrapi(i + 1, nx);
        const int cym = wrapi(j - 1, ny) * nx + wrapi(i, nx), cyp = wrapi(j + 1, ny) * nx + wrapi(i, nx);
        // one lean segment [qa, qb).  phi^n is pure liquid there (the map says so), hence
        // phi^{n+1} = e_l without reading phi^n; it is stored only where the destination's own map
        // does not already show a pure-liquid tile plane (the destination holds phi^{n-1}, and a
        // plane that stayed liquid needs no store).  Register slots hold LD planes of mu in flight
        // (the cell and its four in-plane neighbours); plane q is computed from slot q mod LD,
        // whose loads for plane q+LD are issued right after.  Loads past the segment read clamped
        // planes and are not used.
        // A tile row is one warp, and every lane holds the periodic image of its column (lanes
        // past a ragged edge included), so the x neighbours are the adjacent lanes' cells; only
        // lane 0 (x - 1) and lane TX - 1 (x + 1) load theirs.
        static_assert(TX == 32, "a tile row must be one warp");
        const bool xedge = tx == 0 || tx == TX - 1;
        const int cxe = tx == 0 ? cxm : cxp;
        auto lean = [&](int qa, int qb) {
            constexpr int LD = 8;
            Mu<R> mo[LD], mxe[LD], mym[LD], myp[LD];
            auto load = [&](int u, int k) {
                const size_t o = (size_t)splane(k) * plane;
                mo[u] = ldg_mu(mu + o + col_own);
                if (xedge) mxe[u] = ldg_mu(mu + o + cxe);
                mym[u] = ldg_mu(mu + o + cym);
                myp[u] = ldg_mu(mu + o + cyp);
            };
#pragma unroll
            for (int u = 0; u < LD; u++) load(u, qa + u);
            Ph<R> liquid;
            liquid.v[0] = liquid.v[1] = liquid.v[2] = R(0);
            liquid.v[3] = R(1);
            Mu<R> Vz_lo;
            Vz_lo.v[0] = Vz_lo.v[1] = R(0);
            if (qa > 0) Vz_lo = quiet_zflux(kp, ldg_mu(mu + (size_t)splane(qa - 1) * plane + col_own), mo[0]);
            int phi_stores = 0;
            for (int q0 = qa; q0 < qb; q0 += LD) {
#pragma unroll
                for (int u = 0; u < LD; u++) {
                    const int q = q0 + u;
                    if (q < qb) {
                        // mu of plane q+1: the next slot (for u = LD-1 the slot reloaded at u = 0)
                        const Mu<R> m_next = u + 1 < LD ? mo[u + 1] : mo[0];
                        Mu<R> Vz_hi;
                        Vz_hi.v[0] = Vz_hi.v[1] = R(0);
                        if (q < nz - 1) Vz_hi = quiet_zflux(kp, mo[u], m_next);
                        Mu<R> xm, xp;
#pragma unroll
                        for (int c = 0; c < 2; c++) {
                            xm.v[c] = __shfl_up_sync(0xffffffffu, mo[u].v[c], 1);
                            xp.v[c] = __shfl_down_sync(0xffffffffu, mo[u].v[c], 1);
                        }
                        if (tx == 0) xm = mxe[u];
                        if (tx == TX - 1) xp = mxe[u];
                        const Mu<R> out = quiet_mu_cell(kp, tab + q, mo[u], xm, xp, mym[u], myp[u], Vz_lo, Vz_hi);
                        const size_t o = (size_t)splane(q) * plane;
                        const bool store_phi = !tmap_out || tmap_out[map_idx(splane(q), tile, nz)] != 1;
                        phi_stores += store_phi ? 1 : 0;
                        if (valid) {
                            if (store_phi) st_ph(phi_out + o + col_own, liquid);
                            st_mu(mu_out + o + col_own, out);
                            bad = bad | !isfinite(out.v[0] + out.v[1]);
                        }
                        Vz_lo = Vz_hi;
                        if (q + LD <= qb) load(u, q + LD);
                    }
                }
            }
            // every thread has read the destination's map entries of the segment before any is
            // replaced by the new field's
            __syncthreads();
            if (tmap_out)
                for (int q = qa + tid; q < qb; q += NT) tmap_out[map_idx(splane(q), tile, nz)] = 1;
            // mu^n in, mu^{n+1} out (4 words a cell), plus phi^{n+1} where it was stored
            lean_bytes += tile_cells * (double)sizeof(R) * (4.0 * (qb - qa) + 4.0 * phi_stores);
        };
        if (lean_here && lo_end > z0) lean(z0, lo_end);
        if (lean_here && z1 > hi_beg) lean(hi_beg, z1);
        // the general path runs on the planes in between
        z0 = lo_end;
        z1 = hi_beg;
        if (z0 >= z1) {
            epilogue(0.0, bad, lean_bytes);
            return;
        }
    }

    auto mod3 = [](int k) { return k & 3; };  // ring slot of plane k (4 slots; k >= -2)

    // load slots (phi^n on the 2-ring region, mu^n on the 1-ring region), offsets computed once:
    // slot 0 is cell tid of each region (always present), slot 1 is cell tid + NT where it exists
    const bool hasO1 = tid + NT < SN2, hasM1 = tid + NT < SN;
    const int colO0 = wrapi(j0 + tid / SX2 - 2, ny) * nx + wrapi(i0 + tid % SX2 - 2, nx);
    const int colO1 = hasO1 ? wrapi(j0 + (tid + NT) / SX2 - 2, ny) * nx + wrapi(i0 + (tid + NT) % SX2 - 2, nx) : 0;
    const int colM0 = wrapi(j0 + tid / SX - 1, ny) * nx + wrapi(i0 + tid % SX - 1, nx);
    const int colM1 = hasM1 ? wrapi(j0 + (tid + NT) / SX - 1, ny) * nx + wrapi(i0 + (tid + NT) % SX - 1, nx) : 0;
    // the thread's phi cells on the 1-ring region: its tile cell, and a ring cell for tid < NR
    const bool has_ring = tid < NR;
    int o1[2], o2[2];
    o1[0] = t1;
    o2[0] = t2;
    {
        int li = 0, lj = 0;
        if (has_ring) ring_cell<TX, TY>(tid, li, lj);
        o1[1] = (lj + 1) * SX + (li + 1);
        o2[1] = (lj + 2) * SX2 + (li + 2);
    }
    const bool xtra_y = ty == 0;
    const bool xtra_x = ty == 1 % TY && tx < TY;

    Ph<R> pfO0, pfO1;
    Mu<R> pfM0, pfM1;
    // storage offset of logical plane k: planes inside the domain follow each other in the ring,
    // so the offset of k+1 is the offset of k plus one plane (modulo the ring)
    const size_t ring = (size_t)nz * plane;
    auto next_off = [&](int k, size_t off_k) -> size_t {
        if (k < 0 || k >= nz - 1) return plane_off(k + 1, nz, zbase, plane);
        const size_t o = off_k + plane;
        return o >= ring ? o - ring : o;
    };
    int pk = -1000;  // plane whose offset pko holds
    size_t pko = 0;
    auto prefetch = [&](int k) {
        const size_t b = (k == pk + 1) ? next_off(pk, pko) : plane_off(k, nz, zbase, plane);
        pk = k;
        pko = b;
        pfO0 = ldg_ph(phi + b + colO0);
        pfM0 = ldg_mu(mu + b + colM0);
        if (hasO1) pfO1 = ldg_ph(phi + b + colO1);
        if (hasM1) pfM1 = ldg_mu(mu + b + colM1);
    };
    // store the prefetched plane k with its phase codes; returns whether all of this thread's
    // phi^n cells of the plane are pure liquid (reduced over the CTA by the caller's barrier)
    auto commit = [&](int k) -> bool {
        const int so = mod3(k);
        const int c0 = code_fast(pfO0);
        sO[so * SN2 + tid] = pfO0;
        cO[so * SN2 + tid] = (unsigned char)c0;
        sM[so * SN + tid] = pfM0;
        bool liq = c0 == 3;
        if (hasO1) {
            const int c1 = code_fast(pfO1);
            sO[so * SN2 + tid + NT] = pfO1;
            cO[so * SN2 + tid + NT] = (unsigned char)c1;
            liq = liq & (c1 == 3);
        }
        if (hasM1) sM[so * SN + tid + NT] = pfM1;
        return liq;
    };

    // phi face terms of plane q on the 1-ring region (x faces li|li+1, li in [-2, TX], rows
    // [-1, TY]; y faces lj|lj+1, lj in [-2, TY], columns [-1, TX])
    auto phi_faces = [&](int q) {
        const Ph<R> *Ob = sO + mod3(q) * SN2;
        const unsigned char *Cb = cO + mod3(q) * SN2;
        for (int f = tid; f < PFX + PFY; f += NT) {
            int l, r;
            if (f < PFX) {
                l = (f / (TX + 3)) * SX2 + f % (TX + 3) + SX2;  // (li+2) + (lj+2) SX2 with li = f%(TX+3)-2
                r = l + 1;
            } else {
                const int g = f - PFX;
                l = (g / (TX + 2)) * SX2 + g % (TX + 2) + 1;  // li = g%(TX+2)-1, lj = g/(TX+2)-2
                r = l + SX2;
            }
            const int a = Cb[l], b = Cb[r];
            if (a == b && a < 4) {
                Ph<R> z;
                z.v[0] = z.v[1] = z.v[2] = z.v[3] = R(0);
                sF[f] = z;
            } else {
                sF[f] = face_phi(kp, Ob[l], Ob[r]);
            }
        }
    };
    // z face (q | q+1) of the thread's cell s (equal one-hot cells give zero)
    auto zface_phi = [&](int q, int s) -> Ph<R> {
        const int qa = mod3(q) * SN2, qb = mod3(q + 1) * SN2;
        const int a = cO[qa + o2[s]], b = cO[qb + o2[s]];
        if (a == b && a < 4) {
            Ph<R> z;
            z.v[0] = z.v[1] = z.v[2] = z.v[3] = R(0);
            return z;
        }
        return face_phi(kp, sO[qa + o2[s]], sO[qb + o2[s]]);
    };
    // z-face terms of the thread's 1-ring cells live in a 2-slot shared ring indexed by the parity
    // of the face's lower plane; each thread reads back only what it wrote (no barrier needed)
    auto Fz = [&](int q, int s) -> Ph<R> & { return sFz[(q & 1) * SN + o1[s]]; };
    // phi^{n+1}(q) for the thread's cells; `quiet`: the planes q-1..q+1 of phi^n are pure liquid on
    // the 2-ring region, so phi^{n+1} = phi^n there
    bool own_liq = true;  // the thread's tile cell of the last phi^{n+1} plane is pure liquid (or absent)
    auto phi_new_plane = [&](int q, bool quiet) {
        const Ph<R> *Om = sO + mod3(q - 1) * SN2, *Oq = sO + mod3(q) * SN2, *Op = sO + mod3(q + 1) * SN2;
        const unsigned char *Cm = cO + mod3(q - 1) * SN2, *Cq = cO + mod3(q) * SN2, *Cp = cO + mod3(q + 1) * SN2;
        Ph<R> *Nq = sN + mod3(q) * SN;
        unsigned char *CNq = cN + mod3(q) * SN;
        const Mu<R> *Mq = sM + mod3(q) * SN;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            if (s == 1 && tid >= ((NR + 31) / 32) * 32) break;  // the first warps hold the ring cells
            const bool act = s == 0 || has_ring;
            const int c2 = o2[s];
            const Ph<R> P = Oq[c2];
            const int c = Cq[c2];
            Ph<R> out = P;
            int cout = c;
            if (!quiet) {
                const bool bulk = !act || (c < 4 && Cq[c2 - 1] == c && Cq[c2 + 1] == c && Cq[c2 - SX2] == c &&
                                           Cq[c2 + SX2] == c && Cm[c2] == c && Cp[c2] == c);
                if (!__all_sync(0xffffffffu, bulk)) {
                    if (act) {
                        const int li = o1[s] % SX - 1, lj = o1[s] / SX - 1;
                        const PlaneT<R> T = ldg_plane(tab + q);
                        const Ph<R> *fx = sF + (lj + 1) * (TX + 3) + (li + 2);
                        const Ph<R> *fy = sF + PFX + (lj + 1) * (TX + 2) + (li + 1);
                        out = phi_cell(kp, T, P, Oq[c2 - 1], Oq[c2 + 1], Oq[c2 - SX2], Oq[c2 + SX2], Om[c2], Op[c2],
                                       fx[-1], fx[0], fy[0], fy[TX + 2], Fz(q - 1, s), Fz(q, s), Mq[o1[s]]);
                        cout = code_of(out);
                    }
                }
            }
            if (s == 0) own_liq = !valid || cout == 3;
            if (act) {
                Nq[o1[s]] = out;
                CNq[o1[s]] = (unsigned char)cout;
                if (s == 0 && valid && q >= z0 && q < z1)
                    st_ph(phi_out + plane_off(q, nz, zbase, plane) + col_own, out);
            }
        }
    };
    auto copy_plane = [&](int q, int from) {
        const int d = mod3(q) * SN, s0 = mod3(from) * SN;
        for (int r = tid; r < SN; r += NT) {
            sN[d + r] = sN[s0 + r];
            cN[d + r] = cN[s0 + r];
        }
    };

    // mu face fluxes.  L1/L2: the left (lower) cell in the 1-ring / 2-ring layouts.
    auto mu_xface = [&](int q, int L1, int L2) -> Mu<R> {
        const int sq = mod3(q) * SN;
        const Ph<R> *Nq = sN + sq, *Np = sN + mod3(q + 1) * SN, *Nm = sN + mod3(q - 1) * SN;
        const Ph<R> *Oq = sO + mod3(q) * SN2;
        const Mu<R> *Mq = sM + sq;
        return face_mu_coded(kp, tab + q, cN[sq + L1], cN[sq + L1 + 1], Nq[L1], Nq[L1 + 1], Oq[L2], Oq[L2 + 1],
                             Mq[L1], Mq[L1 + 1], Nq[L1 + SX], Nq[L1 - SX], Nq[L1 + 1 + SX], Nq[L1 + 1 - SX], Np[L1],
                             Nm[L1], Np[L1 + 1], Nm[L1 + 1]);
    };
    auto mu_yface = [&](int q, int L1, int L2) -> Mu<R> {
        const int sq = mod3(q) * SN;
        const Ph<R> *Nq = sN + sq, *Np = sN + mod3(q + 1) * SN, *Nm = sN + mod3(q - 1) * SN;
        const Ph<R> *Oq = sO + mod3(q) * SN2;
        const Mu<R> *Mq = sM + sq;
        const int R1 = L1 + SX;
        return face_mu_coded(kp, tab + q, cN[sq + L1], cN[sq + R1], Nq[L1], Nq[R1], Oq[L2], Oq[L2 + SX2], Mq[L1],
                             Mq[R1], Nq[L1 + 1], Nq[L1 - 1], Nq[R1 + 1], Nq[R1 - 1], Np[L1], Nm[L1], Np[R1], Nm[R1]);
    };
    auto mu_zface = [&](int q) -> Mu<R> {
        if (q < 0 || q >= nz - 1) {
            Mu<R> v;
            v.v[0] = v.v[1] = R(0);
            return v;
        }
        const int sq = mod3(q) * SN, sp = mod3(q + 1) * SN;
        const Ph<R> *Nq = sN + sq, *Np = sN + sp;
        return face_mu_coded(kp, tab + nz + q, cN[sq + t1], cN[sp + t1], Nq[t1], Np[t1], sO[mod3(q) * SN2 + t2],
                             sO[mod3(q + 1) * SN2 + t2], sM[sq + t1], sM[sp + t1], Nq[t1 + 1], Nq[t1 - 1], Np[t1 + 1],
                             Np[t1 - 1], Nq[t1 + SX], Nq[t1 - SX], Np[t1 + SX], Np[t1 - SX]);
    };
    // quiet (pure liquid) planes: constant mobility, no anti-trapping current -- the same
    // expressions the coded short form evaluates there
    auto mu_faces = [&](int q, bool) {
        sVx[ty * (TX + 1) + tx] = mu_xface(q, t1 - 1, t2 - 1);
        sVy[ty * TX + tx] = mu_yface(q, t1 - SX, t2 - SX2);
        if (xtra_y) sVy[TY * TX + tx] = mu_yface(q, TY * SX + tx + 1, (TY + 1) * SX2 + tx + 2);
        if (xtra_x) sVx[tx * (TX + 1) + TX] = mu_xface(q, (tx + 1) * SX + TX, (tx + 2) * SX2 + TX + 1);
    };
    auto mu_zflux_quiet = [&](int q) -> Mu<R> {
        Mu<R> v;
        if (q < 0 || q >= nz - 1) {
            v.v[0] = v.v[1] = R(0);
            return v;
        }
        return quiet_zflux(kp, sM[mod3(q) * SN + t1], sM[mod3(q + 1) * SN + t1]);
    };

    double liq_def = 0.0;
    int solid_cells = 0;
    unsigned hist = 0;  // bit i: phi^n plane (newest - i) is pure liquid on the 2-ring region

    // ---- prologue: phi^{n+1} on planes z0-1 and z0, the z flux below z0 ----
    for (int k = z0 - 2; k <= z0; k++) {
        prefetch(k);
        hist = (hist << 1) | (__syncthreads_and(commit(k)) ? 1u : 0u);
    }
    prefetch(z0 + 1);
    bool quiet = (hist & 7u) == 7u;  // planes z0-2..z0: phi^{n+1}(z0-1) = phi^n(z0-1)
    if (!quiet) phi_faces(z0 - 1);
    // (a thread without a ring cell writes only its own tile cell's entries)
    Fz(z0 - 2, 0) = zface_phi(z0 - 2, 0);
    Fz(z0 - 1, 0) = zface_phi(z0 - 1, 0);
    if (has_ring) {
        Fz(z0 - 2, 1) = zface_phi(z0 - 2, 1);
        Fz(z0 - 1, 1) = zface_phi(z0 - 1, 1);
    }
    __syncthreads();
    if (z0 > 0) phi_new_plane(z0 - 1, quiet);
    __syncthreads();
    hist = (hist << 1) | (__syncthreads_and(commit(z0 + 1)) ? 1u : 0u);
    prefetch(z0 + 2);
    quiet = (hist & 7u) == 7u;  // planes z0-1..z0+1
    if (!quiet) phi_faces(z0);
    Fz(z0, 0) = zface_phi(z0, 0);  // z0-1 | z0 is already in the ring
    if (has_ring) Fz(z0, 1) = zface_phi(z0, 1);
    __syncthreads();
    phi_new_plane(z0, quiet);
    {
        // the barrier also gives the liquid-map entry of phi^{n+1}(z0)
        const int liq_z0 = __syncthreads_and(own_liq);
        if (tmap_out && tid == 0) tmap_out[map_idx(splane(z0), tile, nz)] = liq_z0 ? 1 : 0;
    }
    if (z0 == 0) {
        copy_plane(-1, 0);  // the mirror plane below the domain
        __syncthreads();
    }
    Mu<R> Vz_lo = mu_zface(z0 - 1);
    __syncthreads();  // phi^n / mu^n plane z0-1 is replaced by the first commit below

    // ---- main loop over planes ----
    for (int q = z0; q < z1; ++q) {
        // S0: plane q+2 of phi^n / mu^n; the CTA-wide pure-liquid flag comes with the barrier
        const bool liq = commit(q + 2);
        prefetch(q + 3);
        hist = (hist << 1) | (__syncthreads_and(liq) ? 1u : 0u);
        const bool phi_quiet = (hist & 7u) == 7u;   // phi^n planes q..q+2
        const bool mu_quiet = (hist & 31u) == 31u;  // phi^n planes q-2..q+2
        // S1: phi faces of plane q+1 and the z faces (q+1 | q+2) of the thread's cells
        if (!phi_quiet) phi_faces(q + 1);
        if (phi_quiet) {
            // both phi^n planes are pure liquid here: the z face terms are exactly zero
            Ph<R> z;
            z.v[0] = z.v[1] = z.v[2] = z.v[3] = R(0);
            Fz(q + 1, 0) = z;
            if (has_ring) Fz(q + 1, 1) = z;
        } else {
            Fz(q + 1, 0) = zface_phi(q + 1, 0);
            if (has_ring) Fz(q + 1, 1) = zface_phi(q + 1, 1);
        }
        // a quiet phi plane computes no faces: S2 does not wait for S1
        if (!phi_quiet) __syncthreads();
        // S2: phi^{n+1}(q+1) (a copy of plane nz-1 above the domain)
        if (q + 1 < nz)
            phi_new_plane(q + 1, phi_quiet);
        else
            copy_plane(q + 1, q);
        if (mu_quiet) {
            // S3+S4 of a pure-liquid plane: the flux of a face is one subtraction and two products,
            // so each cell evaluates its four in-plane faces from mu^n directly (both cells of a face
            // evaluate the same expression: the result is that of the staged faces) -- no barrier
            // (phi^{n+1}(q+1) = phi^n(q+1) is pure liquid on the tile: its liquid-map entry is 1)
            if (tmap_out && tid == 0 && q + 1 < z1) tmap_out[map_idx(splane(q + 1), tile, nz)] = 1;
            const Mu<R> *Mq = sM + mod3(q) * SN;
            const Mu<R> mP = Mq[t1];
            const Mu<R> Vz_hi = mu_zflux_quiet(q);
            const Mu<R> out = quiet_mu_cell(kp, tab + q, mP, Mq[t1 - 1], Mq[t1 + 1], Mq[t1 - SX], Mq[t1 + SX], Vz_lo,
                                            Vz_hi);
            if (valid) {
                st_mu(mu_out + plane_off(q, nz, zbase, plane) + col_own, out);
                bad = bad | !isfinite(out.v[0] + out.v[1]);
            }
            Vz_lo = Vz_hi;
            continue;
        }
        {
            // S3 reads phi^{n+1}(q+1) written by other threads in S2; the barrier also gives the
            // liquid-map entry of that plane
            const int liq_q1 = __syncthreads_and(phi_quiet || own_liq);
            if (tmap_out && tid == 0 && q + 1 < z1) tmap_out[map_idx(splane(q + 1), tile, nz)] = liq_q1 ? 1 : 0;
        }
        // S3: mu face fluxes of plane q, the z flux (q | q+1)
        mu_faces(q, false);
        const Mu<R> Vz_hi = mu_zface(q);
        const int sq1 = mod3(q) * SN;
        const Mu<R> mP = sM[sq1 + t1];
        const Ph<R> nP = sN[sq1 + t1], oP = sO[mod3(q) * SN2 + t2];
        const int cn = cN[sq1 + t1], co = cO[mod3(q) * SN2 + t2];
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
                if (cn != 3) {
                    if (cn < 3)
                        solid_cells++;
                    else
                        liq_def += 1.0 - (double)nP.v[3];
                }
                // a non-finite phi^{n+1} reaches mu^{n+1} through h (such a cell is never quiet)
                bad = bad | !isfinite(out.v[0] + out.v[1]);
            }
        }
        Vz_lo = Vz_hi;
    }

    // general planes: phi^n, mu^n in, phi^{n+1}, mu^{n+1} out (12 words a cell)
    epilogue(liq_def + (double)solid_cells, bad, lean_bytes + tile_cells * (double)sizeof(R) * 12.0 * (z1 - z0));
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, sizeof(R) == 4 ? 2 : 1) fused_step_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi,
                                                           const Mu<R> *__restrict__ mu,
                                                           Ph<R> *__restrict__ phi_out, Mu<R> *__restrict__ mu_out,
                                                           const DevState *__restrict__ st,
                                                           const PlaneT<R> *__restrict__ tab,
                                                           Partial *__restrict__ partials,
                                                           const unsigned char *__restrict__ tmap_in,
                                                           unsigned char *__restrict__ tmap_out, int lean_here)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    fused_tile<R, TX, TY>(kp, phi, mu, phi_out, mu_out, st, tab, partials + bid, blockIdx.x, blockIdx.y, blockIdx.z,
                          smem_raw, tmap_in, tmap_out, lean_here != 0);
}

// The general planes of a fused step whose lean planes run in lean_step_kernel: persistent CTAs
// take the (tile, chunk) items that plan_kernel listed, one at a time, and run the general path on
// each item's precomputed range.
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, sizeof(R) == 4 ? 2 : 1) general_step_kernel(
    const KParams<R> kp, const Ph<R> *__restrict__ phi, const Mu<R> *__restrict__ mu, Ph<R> *__restrict__ phi_out,
    Mu<R> *__restrict__ mu_out, const DevState *__restrict__ st, const PlaneT<R> *__restrict__ tab,
    Partial *__restrict__ partials, const unsigned char *__restrict__ tmap_in, unsigned char *__restrict__ tmap_out,
    const int2 *__restrict__ splits, const int *__restrict__ glist, LeanStats *__restrict__ stats)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int ntl = kp.tgx * kp.tgy;
    for (;;) {
        __syncthreads();  // the previous item is done with s_item and the shared rings
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(&stats->gnext, 1u);
            s_item = it < *(volatile unsigned *)&stats->gcount ? glist[it] : -1;
        }
        __syncthreads();
        const int item = s_item;
        if (item < 0) break;
        const int bz = item / ntl, tile = item % ntl;
        fused_tile<R, TX, TY>(kp, phi, mu, phi_out, mu_out, st, tab, partials + item, tile % kp.tgx, tile / kp.tgx,
                              bz, smem_raw, tmap_in, tmap_out, false, splits + item);
    }
}

// The general planes as the two sweeps: persistent CTAs take the listed (tile, chunk) items one
// at a time (phi pass: counter gnext, mu pass: gnext_mu) and sweep each item's general range.
// Registers are budgeted for PF_GENERAL_MIN_CTAS resident CTAs per SM (2: ~100 registers; 3 fits 80
// registers without spills but ran slower on the 256x256x1024 workload).
#ifndef PF_GENERAL_MIN_CTAS
#define PF_GENERAL_MIN_CTAS 2
#endif
// PF_GENERAL_MAXNREG > 0: the single-domain general kernels take that register cap instead (so that
// lean CTAs fit beside two general CTAs on an SM)
#if defined(PF_GENERAL_MAXNREG) && PF_GENERAL_MAXNREG > 0
#define PF_GENERAL_BOUNDS(n) __maxnreg__(PF_GENERAL_MAXNREG)
#else
#define PF_GENERAL_BOUNDS(n) __launch_bounds__(n, PF_GENERAL_MIN_CTAS)
#endif
template <typename R, int TX, int TY, bool SYM, bool COMP = false>
__global__ void PF_GENERAL_BOUNDS(TX *TY) general_phi_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi,
                                                            const Mu<R> *__restrict__ mu, Ph<R> *__restrict__ phi_out,
                                                            const DevState *__restrict__ st,
                                                            const PlaneT<R> *__restrict__ tab,
                                                            const unsigned char *__restrict__ tmap_in,
                                                            unsigned char *__restrict__ tmap_out,
                                                            const int2 *__restrict__ splits,
                                                            const int *__restrict__ glist,
                                                            LeanStats *__restrict__ stats, int slots,
                                                            int after_lean, const Ph<R> *__restrict__ phi_lo,
                                                            Ph<R> *__restrict__ phi_out_lo)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    // after_lean: the kernel ahead of this one in the stream is the lean kernel of the same step, whose
    // CTAs all passed their wait for the plan before this kernel could be scheduled.  This sweep reads
    // nothing the lean kernel writes (other planes, other map entries), so it starts as lean CTAs retire
    // and waits for the lean kernel only before it exits (its own completion then still implies the
    // lean kernel's).  Any other predecessor is waited for first: the plan's list must be complete.
    if (!after_lean) pdl_wait();
    pdl_trigger();
    const int ntl = kp.tgx * kp.tgy;
    const unsigned G = __ldcg(&stats->gcount);
    const int U = general_units(G, slots);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(&stats->gnext, 1u);
            s_item = it < G * (unsigned)U ? (int)it : -1;
        }
        __syncthreads();
        const int entry = s_item;
        if (entry < 0) break;
        const int item = __ldcg(glist + entry / U), unit = entry % U, tile = item % ntl;
        const int2 sp = __ldcg(splits + item);
        int za, zb;
        unit_range(sp.x, sp.y, U, unit, za, zb);
        if (za < zb)
            phi_sweep_tile<R, TX, TY, COMP, SYM>(kp, phi, mu, phi_out, st, tab, phi_lo, phi_out_lo, tile % kp.tgx,
                                                 tile / kp.tgx, za, zb, smem_raw, tmap_out, tmap_in,
                                                 &stats->map_changed);
    }
    pdl_wait();
}
template <typename R, int TX, int TY, bool SYM, bool COMP = false>
__global__ void PF_GENERAL_BOUNDS(TX *TY) general_mu_kernel(const KParams<R> kp, const Ph<R> *__restrict__ phi_old,
                                                           const Ph<R> *__restrict__ phi_new,
                                                           const Mu<R> *__restrict__ mu, Mu<R> *__restrict__ mu_out,
                                                           const DevState *__restrict__ st,
                                                           const PlaneT<R> *__restrict__ tab,
                                                           Partial *__restrict__ partials,
                                                           const int2 *__restrict__ splits,
                                                           const int *__restrict__ glist,
                                                           LeanStats *__restrict__ stats,
                                                           Partial *__restrict__ subparts,
                                                           unsigned *__restrict__ subcnt, int slots,
                                                           const Mu<R> *__restrict__ mu_lo,
                                                           Mu<R> *__restrict__ mu_out_lo)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    pdl_wait();  // phi^{n+1} of the phi-sweep (and, through its own wait, the lean kernel)
    pdl_trigger();
    const int ntl = kp.tgx * kp.tgy;
    const unsigned G = __ldcg(&stats->gcount);
    const int U = general_units(G, slots);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(&stats->gnext_mu, 1u);
            s_item = it < G * (unsigned)U ? (int)it : -1;
        }
        __syncthreads();
        const int entry = s_item;
        if (entry < 0) break;
        const int item = glist[entry / U], unit = entry % U, tile = item % ntl;
        const int2 sp = splits[item];
        int za, zb;
        unit_range(sp.x, sp.y, U, unit, za, zb);
        // both sweeps' compulsory words: phi^n, mu^n in, phi^{n+1} out; phi^n, phi^{n+1}, mu^n in,
        // mu^{n+1} out.  An item of one unit writes its partial directly; otherwise each unit writes
        // its own (an empty unit a zero one) and the item's last unit to finish sums them in unit
        // order (a fixed order, so the FP64 sums do not depend on which unit finishes last).
        Partial *mine = U == 1 ? partials + item : subparts + (size_t)item * kMaxUnits + unit;
        // (the compensated state adds the low words of phi in and out, of mu in and out: 34 words)
        if (za < zb)
            mu_sweep_tile<R, TX, TY, COMP, SYM>(kp, phi_old, phi_new, mu, mu_out, st, tab, mine, mu_lo, mu_out_lo,
                                                tile % kp.tgx, tile / kp.tgx, za, zb, smem_raw, COMP ? 34.0 : 22.0,
                                                splits, kp.zchunk);
        else if (threadIdx.x == 0)
            zero_partial(mine);
        if (U > 1 && threadIdx.x == 0) {
            __threadfence();  // this unit's partial is visible before its arrival is counted
            const unsigned done = atomicAdd(subcnt + item, 1u);
            if (done == (unsigned)(U - 1)) {
                __threadfence();
                Partial sum;
                sum.liq_deficit = sum.nonfinite = sum.bytes = sum.timeout = 0.0;
                for (int u = 0; u < U; u++) {
                    const volatile Partial *q = subparts + (size_t)item * kMaxUnits + u;
                    sum.liq_deficit += q->liq_deficit;
                    sum.nonfinite += q->nonfinite;
                    sum.bytes += q->bytes;
                    sum.timeout += q->timeout;
                }
                partials[item] = sum;
                subcnt[item] = 0u;  // ready for the next step
            }
        }
    }
}

// Plan of a batched step: four (domain, item) entries of the table per CTA; general items are
// appended to the batch-wide list.  PLAN_PER_BATCH planes per thread cover z chunks up to 572.
constexpr int PLAN_PER_BATCH = 9;
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(256) batched_plan_kernel(const BatchDomain<R> *__restrict__ doms,
                                                           const int2 *__restrict__ entries, int nentries,
                                                           int parity, int2 *__restrict__ glist,
                                                           BatchPlan *__restrict__ plan)
{
    __shared__ int kred[8][2];
    const int e = blockIdx.x * 4 + (threadIdx.x >> 6);
    const bool live = e < nentries;
    const int2 en = live ? entries[e] : make_int2(0, 0);
    const BatchDomain<R> *d = doms + en.x;
    int lo_end, hi_beg;
    plan_item<TX, TY, PLAN_PER_BATCH>(d->kp.nx, d->kp.ny, d->kp.nz, d->kp.tgx, d->kp.tgy, d->kp.zchunk, d->st->zbase,
                                      d->tmap[parity], en.y, live, kred, lo_end, hi_beg);
    if (live && (threadIdx.x & 63) == 0) {
        d->splits[en.y] = make_int2(lo_end, hi_beg);
        if (hi_beg > lo_end)
            glist[atomicAdd(&plan->gcount, 1u)] = en;
        else
            zero_partial(d->parts + en.y);
    }
}

// The general planes of a batched step as the two sweeps: persistent CTAs over the batch-wide list
// of (domain, item) entries (pass 0: phi-sweep, counter gnext; pass 1: mu-sweep, counter gnext_mu).
// SYM: every domain of the batch has the symmetric set (the instantiation without the general-
// thermodynamics branches, as the single-domain general kernels).
template <typename R, int TX, int TY, int PASS, bool SYM>
__global__ void __launch_bounds__(TX *TY, PF_GENERAL_MIN_CTAS) batched_general_kernel(
    const BatchDomain<R> *__restrict__ doms, const int2 *__restrict__ glist, BatchPlan *__restrict__ plan, int parity)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int2 s_en;
    __shared__ __align__(16) KParams<R> s_kp;
    for (;;) {
        __syncthreads();  // the previous entry's readers of s_kp and shared memory are done
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(PASS == 0 ? &plan->gnext : &plan->gnext_mu, 1u);
            s_en = it < *(volatile unsigned *)&plan->gcount ? glist[it] : make_int2(-1, 0);
        }
        __syncthreads();
        const int2 en = s_en;
        if (en.x < 0) break;
        const BatchDomain<R> *d = doms + en.x;
        {
            const int *src = reinterpret_cast<const int *>(&d->kp);
            int *dst = reinterpret_cast<int *>(&s_kp);
            for (int q = threadIdx.x; q < (int)(sizeof(KParams<R>) / sizeof(int)); q += TX * TY) dst[q] = src[q];
        }
        __syncthreads();
        const int ntl = s_kp.tgx * s_kp.tgy, tile = en.y % ntl;
        const int2 sp = d->splits[en.y];
        const int a = parity, b = parity ^ 1;
        if (PASS == 0)
            phi_sweep_tile<R, TX, TY, false, SYM>(s_kp, (const Ph<R> *)d->phi[a], (const Mu<R> *)d->mu[a], (Ph<R> *)d->phi[b],
                                             d->st, d->tab, nullptr, nullptr, tile % s_kp.tgx, tile / s_kp.tgx, sp.x,
                                             sp.y, smem_raw, d->tmap[b]);
        else
            mu_sweep_tile<R, TX, TY, false, SYM>(s_kp, (const Ph<R> *)d->phi[a], (const Ph<R> *)d->phi[b],
                                            (const Mu<R> *)d->mu[a], (Mu<R> *)d->mu[b], d->st, d->tab,
                                            d->parts + en.y, nullptr, nullptr, tile % s_kp.tgx, tile / s_kp.tgx, sp.x,
                                            sp.y, smem_raw, 22.0, d->splits, s_kp.zchunk);
    }
}

// ---------------------------------------------------------------------------------------
// batched step: many independent domains of uneven size in one persistent launch.  Each CTA
// pulls (domain, tile, z chunk) work items from a table through an atomic counter (largest
// chunks first in the table), copies that domain's parameters into shared memory and runs the
// same tile body as the single-domain kernel.
// ---------------------------------------------------------------------------------------
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, sizeof(R) == 4 ? 2 : 1) batched_fused_kernel(const BatchDomain<R> *__restrict__ doms,
                                                              const BatchItem *__restrict__ items, int nitems,
                                                              unsigned *__restrict__ counter, int parity)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ __align__(16) KParams<R> s_kp;
    for (;;) {
        __syncthreads();  // the previous item's readers of s_kp and shared memory are done
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const BatchItem w = items[it];
        const BatchDomain<R> *d = doms + w.dom;
        {
            const int *src = reinterpret_cast<const int *>(&d->kp);
            int *dst = reinterpret_cast<int *>(&s_kp);
            for (int q = threadIdx.x; q < (int)(sizeof(KParams<R>) / sizeof(int)); q += TX * TY) dst[q] = src[q];
        }
        __syncthreads();
        const int a = parity, b = parity ^ 1;
        Partial *part = d->parts + ((size_t)w.bz * d->gy + w.by) * d->gx + w.bx;
        fused_tile<R, TX, TY>(s_kp, (const Ph<R> *)d->phi[a], (const Mu<R> *)d->mu[a], (Ph<R> *)d->phi[b],
                              (Mu<R> *)d->mu[b], d->st, d->tab, part, w.bx, w.by, w.bz, smem_raw, d->tmap[a],
                              d->tmap[b]);
    }
}

}  // namespace pf
#include "pf_lean.cuh"
#include "pf_mesh.cuh"
namespace pf {

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
__device__ __forceinline__ void finalize_body(const KParams<R> &kp, DevState *__restrict__ st,
                                              const Partial *__restrict__ parts, int nparts,
                                              LeanStats *__restrict__ lean = nullptr)
{
    __shared__ double sa[256], sb[256];
    __shared__ int s_to;
    if (threadIdx.x == 0) s_to = 0;
    __syncthreads();
    double a = 0.0, b = 0.0;
    bool to = false;
#pragma unroll 4
    for (int q = threadIdx.x; q < nparts; q += 256) {
        a += parts[q].liq_deficit;
        b += parts[q].nonfinite;
        to = to || parts[q].timeout > 0.0;
    }
    if (to) atomicOr(&s_to, 1);
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
        bool bad = sb[0] > 0.0, tmo = s_to != 0;
        if (lean) {  // the lean kernel's flags and bytes of this step
            bad = bad || lean->nonfinite != 0;
            tmo = tmo || lean->timeout != 0;
            lean->last_bytes = lean->bytes;
            lean->bytes = 0ull;
            lean->nonfinite = 0;
            lean->timeout = 0;
            lean->gnext = 0u;
            lean->gnext_mu = 0u;
        }
        if (bad && st->nonfinite == 0) st->nonfinite = 1;
        if (tmo) st->nonfinite = 2;
        const double h = sa[0] / ((double)kp.nx * (double)kp.ny);
        st->h_int = h;
        st->liq = sa[0];
        int s = 0;
        if (kp.window && h >= kp.window_trigger_z) {
            s = (int)floor(h - kp.window_trigger_z) + 1;
            if (s > kp.nz - 1) s = kp.nz - 1;
            if (s < 0) s = 0;
        }
        st->shift = s;
        if (lean) {
            // the plan of this step still holds for the new field unless a liquid-map entry changed or
            // the window moves; otherwise the next plan kernel lists the items afresh
            const int valid = lean->map_changed == 0 && s == 0 ? 1 : 0;
            lean->plan_valid = valid;
            if (!valid) lean->gcount = 0u;
            lean->map_changed = 0;
        }
        if (s > 0) {
            int zb = st->zbase + s;
            if (zb >= kp.nz) zb -= kp.nz;
            st->zbase = zb;
            st->off = st->off + (double)s;
            st->nshift_total += s;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) finalize_kernel(const KParams<R> kp, DevState *__restrict__ st,
                                                      const Partial *__restrict__ parts, int nparts,
                                                      LeanStats *__restrict__ lean)
{
    pdl_wait();
    pdl_trigger();
    finalize_body(kp, st, parts, nparts, lean);
}

// one block per domain
template <typename R>
__global__ void __launch_bounds__(256) batched_finalize_kernel(const BatchDomain<R> *__restrict__ doms)
{
    const BatchDomain<R> *d = doms + blockIdx.x;
    finalize_body(d->kp, d->st, d->parts, d->gx * d->gy * d->gz, d->lean);
}

// After finalize: rebuild the plane table for the new (t, offset) and fill the planes that
// entered the window (phi = liquid, mu = the previous top plane's mu).
template <typename R>
__device__ __forceinline__ void post_body(const KParams<R> &kp, const DevState *__restrict__ st,
                                          Ph<R> *__restrict__ phi, Mu<R> *__restrict__ mu,
                                          PlaneT<R> *__restrict__ tab, Ph<R> *__restrict__ phi_lo,
                                          Mu<R> *__restrict__ mu_lo, size_t tid, size_t nth,
                                          unsigned char *__restrict__ tmap)
{
    const double t = st->t, off = st->off;
    const int s = st->shift, zbase = st->zbase;
    const int nz = kp.nz;
    for (size_t e = tid; e < (size_t)2 * nz; e += nth) {
        if (e < (size_t)nz)
            make_plane(kp, (double)e + off, t, tab + e);
        else
            make_plane(kp, ((double)(e - nz) + off) + 0.5, t, tab + e);
    }
    if (s > 0 && tmap) {
        // the entering planes are pure liquid, and so is their liquid-map entry
        const size_t ntl = (size_t)kp.tgx * kp.tgy;
        for (size_t q = tid; q < (size_t)s * ntl; q += nth) {
            int sp = nz - s + (int)(q / ntl) + zbase;
            if (sp >= nz) sp -= nz;
            tmap[map_idx(sp, (int)(q % ntl), nz)] = 1;
        }
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
            if (phi_lo) {
                Ph<R> z;
                z.v[0] = z.v[1] = z.v[2] = z.v[3] = R(0);
                st_ph(phi_lo + dst, z);
            }
            if (mu_lo) st_mu(mu_lo + dst, mu_lo[src + c]);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) post_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                  Ph<R> *__restrict__ phi, Mu<R> *__restrict__ mu,
                                                  PlaneT<R> *__restrict__ tab, Ph<R> *__restrict__ phi_lo,
                                                  Mu<R> *__restrict__ mu_lo, unsigned char *__restrict__ tmap)
{
    pdl_wait();
    pdl_trigger();
    post_body(kp, st, phi, mu, tab, phi_lo, mu_lo, (size_t)blockIdx.x * blockDim.x + threadIdx.x,
              (size_t)gridDim.x * blockDim.x, tmap);
}

// grid (blocks per domain, domains); the new source fields of each domain are phi/mu[parity ^ 1]
template <typename R>
__global__ void __launch_bounds__(256) batched_post_kernel(const BatchDomain<R> *__restrict__ doms, int parity)
{
    const BatchDomain<R> *d = doms + blockIdx.y;
    post_body(d->kp, d->st, (Ph<R> *)d->phi[parity ^ 1], (Mu<R> *)d->mu[parity ^ 1], d->tab, (Ph<R> *)nullptr,
              (Mu<R> *)nullptr, (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x,
              d->tmap[parity ^ 1]);
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
    // a slab of a decomposed domain takes the rows of the global domain it covers
    const int nyg = kp.gny > 0 ? kp.gny : kp.ny;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / plane);
        const int jl = (int)((q % plane) / kp.nx);
        const int j = kp.gny > 0 ? ((jl + kp.gy0) % nyg + nyg) % nyg : jl;
        const int i = (int)(q % kp.nx);
        int ph = 3;
        if (k < H && n_grains > 0) {
            int best = -1;
            double bestd = 0.0;
            for (int g = 0; g < n_grains; g++) {
                double ddx = fabs(__dadd_rn((double)i + 0.5, -seeds[4 * g + 0]));
                double ddy = fabs(__dadd_rn((double)j + 0.5, -seeds[4 * g + 1]));
                double ddz = fabs(__dadd_rn((double)k + 0.5, -seeds[4 * g + 2]));
                const double wx = __dadd_rn((double)kp.nx, -ddx), wy = __dadd_rn((double)nyg, -ddy);
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
                                                    double *__restrict__ out, const Ph<R> *__restrict__ phi_lo,
                                                    const Mu<R> *__restrict__ mu_lo)
{
    __shared__ double sh[8][256];
    const int k = blockIdx.x;
    const size_t plane = (size_t)kp.nx * kp.ny;
    const size_t base = plane_off(k, kp.nz, st->zbase, plane);
    const double T = kp.T0 + kp.G * (((double)k + st->off) * kp.dx64 - kp.v * st->t);
    double ch[4][2];  // per-plane constants: cE_a + kT_a (T - TE)
    for (int a = 0; a < 4; a++) {
        ch[a][0] = kp.cE[a][0] + kp.kT64[a][0] * (T - kp.TE);
        ch[a][1] = kp.cE[a][1] + kp.kT64[a][1] * (T - kp.TE);
    }
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // a slab of a decomposed domain sums its own rows only
    const size_t q0 = kp.gny > 0 ? (size_t)kp.red_j0 * kp.nx : 0, q1 = kp.gny > 0 ? (size_t)kp.red_j1 * kp.nx : plane;
    for (size_t q = q0 + threadIdx.x; q < q1; q += 256) {
        const Ph<R> p = ldg_ph(phi + base + q);
        const Mu<R> m = ldg_mu(mu + base + q);
        Ph<R> pl;
        Mu<R> ml;
        pl.v[0] = pl.v[1] = pl.v[2] = pl.v[3] = R(0);
        ml.v[0] = ml.v[1] = R(0);
        if (phi_lo) pl = ldg_ph(phi_lo + base + q);
        if (mu_lo) ml = ldg_mu(mu_lo + base + q);
        double ph[4], S = 0.0;
        for (int a = 0; a < 4; a++) {
            ph[a] = (double)p.v[a] + (double)pl.v[a];
            S += ph[a] * ph[a];
        }
        const double m0 = (double)m.v[0] + (double)ml.v[0], m1 = (double)m.v[1] + (double)ml.v[1];
        bool bad = !isfinite(m0) || !isfinite(m1);
        double c0 = 0.0, c1 = 0.0;
        const double iS = 1.0 / S;  // one FP64 division per cell (the FP64 rate is low on this part)
        for (int a = 0; a < 4; a++) {
            bad = bad || !isfinite(ph[a]);
            acc[a] += ph[a];
            const double h = ph[a] * ph[a] * iS;
            // c^a = K_a mu + chat_a (K_a = I/(2 A_a) for the identity form)
            c0 += h * (kp.K64[a][0] * m0 + kp.K64[a][1] * m1 + ch[a][0]);
            c1 += h * (kp.K64[a][1] * m0 + kp.K64[a][2] * m1 + ch[a][1]);
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

// AoS device fields (ring-buffered) <-> SoA staging of the host element type H (double or float) for
// logical planes [k0, k0 + nk).  A compensated state packs the value of its pair (high + low, then
// rounded once to H) and unpacks into a canonical pair.
template <typename R, typename H>
__global__ void __launch_bounds__(256) pack_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                  const Ph<R> *__restrict__ phi, const Mu<R> *__restrict__ mu,
                                                  H *__restrict__ phi_soa, H *__restrict__ mu_soa, int k0, int nk,
                                                  const Ph<R> *__restrict__ phi_lo, const Mu<R> *__restrict__ mu_lo)
{
    const size_t plane = (size_t)kp.nx * kp.ny, n = plane * nk;
    const int zbase = st->zbase;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(q / plane);
        const size_t c = q % plane;
        const size_t g = plane_off(k0 + kk, kp.nz, zbase, plane) + c;
        if (phi_soa) {
            const Ph<R> p = ldg_ph(phi + g);
            double v[4];
            for (int a = 0; a < 4; a++) v[a] = (double)p.v[a];
            if (phi_lo) {
                const Ph<R> l = ldg_ph(phi_lo + g);
                for (int a = 0; a < 4; a++) v[a] += (double)l.v[a];
            }
            for (int a = 0; a < 4; a++) phi_soa[(size_t)a * n + q] = (H)v[a];
        }
        if (mu_soa) {
            const Mu<R> m = ldg_mu(mu + g);
            double v0 = (double)m.v[0], v1 = (double)m.v[1];
            if (mu_lo) {
                const Mu<R> l = ldg_mu(mu_lo + g);
                v0 += (double)l.v[0];
                v1 += (double)l.v[1];
            }
            mu_soa[q] = (H)v0;
            mu_soa[n + q] = (H)v1;
        }
    }
}

template <typename R, typename H>
__global__ void __launch_bounds__(256) unpack_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                    Ph<R> *__restrict__ phi, Mu<R> *__restrict__ mu,
                                                    const H *__restrict__ phi_soa, const H *__restrict__ mu_soa,
                                                    int k0, int nk, Ph<R> *__restrict__ phi_lo,
                                                    Mu<R> *__restrict__ mu_lo)
{
    const size_t plane = (size_t)kp.nx * kp.ny, n = plane * nk;
    const int zbase = st->zbase;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(q / plane);
        const size_t c = q % plane;
        const size_t g = plane_off(k0 + kk, kp.nz, zbase, plane) + c;
        Ph<R> p, pl;
        for (int a = 0; a < 4; a++) {
            const double x = (double)phi_soa[(size_t)a * n + q];
            p.v[a] = (R)x;
            pl.v[a] = (R)(x - (double)p.v[a]);
        }
        st_ph(phi + g, p);
        if (phi_lo) st_ph(phi_lo + g, pl);
        Mu<R> m, ml;
        for (int c = 0; c < 2; c++) {
            const double x = (double)mu_soa[(size_t)c * n + q];
            m.v[c] = (R)x;
            ml.v[c] = (R)(x - (double)m.v[c]);
        }
        st_mu(mu + g, m);
        if (mu_lo) st_mu(mu_lo + g, ml);
    }
}

// Liquid map of a field: one byte per (storage plane, fused-step tile), 1 when every cell of the
// tile in that plane is exactly pure liquid.  Grid (tiles, groups of 32 planes).
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) classify_kernel(const KParams<R> kp, const DevState *__restrict__ st,
                                                         const Ph<R> *__restrict__ phi,
                                                         unsigned char *__restrict__ tmap,
                                                         const Ph<R> *__restrict__ phi_lo)
{
    const int tile = blockIdx.x, bx = tile % kp.tgx, by = tile / kp.tgx;
    const int i = bx * TX + (int)threadIdx.x % TX, j = by * TY + (int)threadIdx.x / TX;
    const bool valid = i < kp.nx && j < kp.ny;
    const size_t plane = (size_t)kp.nx * kp.ny;
    const int zbase = st->zbase;
    const int k0 = blockIdx.y * 32, k1 = min(k0 + 32, kp.nz);
    for (int k = k0; k < k1; k++) {
        const size_t off = plane_off(k, kp.nz, zbase, plane);
        bool liq = !valid || code_of(ldg_ph(phi + off + (size_t)j * kp.nx + i)) == 3;
        if (phi_lo && valid) {  // a compensated state is exactly pure liquid with zero low words only
            const Ph<R> l = ldg_ph(phi_lo + off + (size_t)j * kp.nx + i);
            liq = liq && l.v[0] == R(0) && l.v[1] == R(0) && l.v[2] == R(0) && l.v[3] == R(0);
        }
        const int all = __syncthreads_and(liq);
        if (threadIdx.x == 0) tmap[map_idx((int)(off / plane), tile, kp.nz)] = all ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
constexpr int kTX = 32, kTY = 8;

// A set-up done once per device: a kernel's maximum dynamic shared memory is a per-device setting, so
// every device that launches the kernel needs it.  done() tells whether the current device has been
// set up, mark() records it.  Safe across host threads (two threads may both run the idempotent
// set-up once); a device index beyond the table runs the set-up on every launch.
struct DeviceOnce {
    static constexpr int kMax = 64;
    std::atomic<bool> flag[kMax] = {};
    static int device()
    {
        int d = -1;
        if (cudaGetDevice(&d) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        return d;
    }
    bool done() const
    {
        const int d = device();
        return d >= 0 && d < kMax && flag[d].load(std::memory_order_acquire);
    }
    void mark()
    {
        const int d = device();
        if (d >= 0 && d < kMax) flag[d].store(true, std::memory_order_release);
    }
};


// Launch of kernel k with the programmatic stream serialisation attribute when pdl is set (the kernel
// may then be scheduled while the one ahead of it in the stream is still running; it calls pdl_wait()
// before it depends on that kernel's results), a plain launch otherwise.
// prio: with the device's highest priority (kept in a captured graph's kernel node), so that the
// launch's CTAs are placed before those of a concurrent launch of lower priority.
template <typename... KArgs, typename... Args>
static cudaError_t launch_kp(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                             bool prio, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        na++;
    }
    if (prio) {
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess) {
            at[na].id = cudaLaunchAttributePriority;
            at[na].val.priority = hi;
            na++;
        }
    }
    cfg.attrs = na ? at : nullptr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                            Args &&...args)
{
    return launch_kp(k, grid, block, smem, s, pdl, false, std::forward<Args>(args)...);
}

template <typename R>
static size_t phi_smem_bytes()
{
    constexpr int SN = (kTX + 2) * (kTY + 2), FX = kTY * (kTX + 1), FY = (kTY + 1) * kTX, NS = phi_ring<R>();
    return sizeof(Ph<R>) * (NS * SN + 2 * FX + 2 * FY) + sizeof(Mu<R>) * NS * kTX * kTY;
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
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = phi_smem_bytes<R>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(phi_sweep_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
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
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = mu_smem_bytes<R>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(mu_sweep_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
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
    return sizeof(Ph<R>) * (4 * SN2 + 4 * SN + PFX + PFY + 2 * SN) + sizeof(Mu<R>) * (4 * SN + FX + FY) + 4 * SN2 +
           4 * SN;
}

template <typename R>
cudaError_t launch_classify(const KParams<R> &kp, const DevState *st, const void *phi, unsigned char *tmap,
                            cudaStream_t s, const void *phi_lo)
{
    if (kp.tgx * kTX < kp.nx || kp.tgy * kTY < kp.ny) return cudaErrorInvalidValue;
    dim3 grid(kp.tgx * kp.tgy, (kp.nz + 31) / 32);
    classify_kernel<R, kTX, kTY><<<grid, kTX * kTY, 0, s>>>(kp, st, (const Ph<R> *)phi, tmap, (const Ph<R> *)phi_lo);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fused_step(const KParams<R> &kp, const Geometry &g, const void *phi, const void *mu,
                              void *phi_out, void *mu_out, const DevState *st, const PlaneT<R> *tab, Partial *parts,
                              cudaStream_t s, const unsigned char *tmap_in, unsigned char *tmap_out, bool lean_here)
{
    if ((tmap_in || tmap_out) && (kp.tgx != g.gx || kp.tgy != g.gy)) return cudaErrorInvalidValue;
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = fused_smem_bytes<R>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    dim3 grid(g.gx, g.gy, g.gz);
    fused_step_kernel<R, kTX, kTY><<<grid, kTX * kTY, sm, s>>>(kp, (const Ph<R> *)phi, (const Mu<R> *)mu,
                                                               (Ph<R> *)phi_out, (Mu<R> *)mu_out, st, tab, parts,
                                                               tmap_in, tmap_out, lean_here ? 1 : 0);
    return cudaGetLastError();
}

// lean kernel shape: pipeline stages, at most planes per CTA, tile rows per consumer thread
#ifndef PF_LEAN_STAGES
#define PF_LEAN_STAGES 8
#endif
#ifndef PF_LEAN_PLANES
#define PF_LEAN_PLANES 64
#endif
#ifndef PF_LEAN_ROWS
#define PF_LEAN_ROWS 4
#endif
constexpr int kLeanStages = PF_LEAN_STAGES, kLeanMaxSub = PF_LEAN_PLANES, kLeanRows = PF_LEAN_ROWS;
// rows a consumer warp owns in the half-height (32 x kTY/2) lean tile of a batched step
constexpr int kLeanRowsHalf = PF_LEAN_ROWS < kTY / 2 ? PF_LEAN_ROWS : kTY / 2;

template <typename R>
cudaError_t launch_plan(const KParams<R> &kp, const Geometry &g, const DevState *st, const unsigned char *tmap_in,
                        int2 *splits, int *glist, LeanStats *stats, Partial *parts, cudaStream_t s, bool pdl)
{
    if (kp.tgx != g.gx || kp.tgy != g.gy) return cudaErrorInvalidValue;
    if (kp.zchunk + 4 > 64 * PLAN_PER) return cudaErrorInvalidValue;
    const int items = g.gx * g.gy * g.gz;
    return launch_k(plan_kernel<kTX, kTY>, dim3((items + 3) / 4), dim3(256), 0, s, pdl, kp.nx, kp.ny, kp.nz, kp.tgx,
                    kp.tgy, kp.zchunk, g.gz, st, tmap_in, splits, glist, stats, parts);
}

template <typename R>
cudaError_t launch_general_step(const KParams<R> &kp, const void *phi, const void *mu, void *phi_out, void *mu_out,
                                const DevState *st, const PlaneT<R> *tab, Partial *parts,
                                const unsigned char *tmap_in, unsigned char *tmap_out, const int2 *splits,
                                const int *glist, LeanStats *stats, int ctas, cudaStream_t s)
{
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = fused_smem_bytes<R>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(general_step_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    general_step_kernel<R, kTX, kTY><<<ctas, kTX * kTY, sm, s>>>(kp, (const Ph<R> *)phi, (const Mu<R> *)mu,
                                                                (Ph<R> *)phi_out, (Mu<R> *)mu_out, st, tab, parts,
                                                                tmap_in, tmap_out, splits, glist, stats);
    return cudaGetLastError();
}

// Dynamic shared memory of the general planes' phi-sweep (the compensated state adds a ring of its
// low words)
template <typename R, bool COMP>
static size_t general_phi_smem_bytes()
{
    return phi_smem_bytes<R>() + (COMP ? sizeof(Ph<R>) * phi_ring<R>() * kTX * kTY : 0);
}
// Dynamic shared memory limits of one instantiation of the general planes' sweeps (SYM: the symmetric
// set, COMP: compensated FP32), and the largest shared-memory carveout (so that as many CTAs as the
// registers allow fit beside each other)
template <typename R, bool SYM, bool COMP>
static cudaError_t general_sweep_attributes_of()
{
    const void *kphi = (const void *)general_phi_kernel<R, kTX, kTY, SYM, COMP>;
    const void *kmu = (const void *)general_mu_kernel<R, kTX, kTY, SYM, COMP>;
    cudaError_t e = cudaFuncSetAttribute(kphi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)general_phi_smem_bytes<R, COMP>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kmu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mu_smem_bytes<R>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kphi, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kmu, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}
template <typename R>
static cudaError_t general_sweep_attributes()
{
    cudaError_t e = general_sweep_attributes_of<R, false, false>();
    if (e == cudaSuccess) e = general_sweep_attributes_of<R, true, false>();
    if constexpr (sizeof(R) == 4)
        if (e == cudaSuccess) e = general_sweep_attributes_of<R, false, true>();
    return e;
}

template <typename R, bool SYM, bool COMP>
static cudaError_t launch_general_pair(const KParams<R> &kp, const void *phi, const void *mu, void *phi_out,
                                       void *mu_out, const DevState *st, const PlaneT<R> *tab, Partial *parts,
                                       const unsigned char *tmap_in, unsigned char *tmap_out, const int2 *splits,
                                       const int *glist, LeanStats *stats, int phi_ctas, int mu_ctas, cudaStream_t s,
                                       Partial *subparts, unsigned *subcnt, bool pdl, bool after_lean,
                                       const void *phi_lo, void *phi_out_lo, const void *mu_lo, void *mu_out_lo,
                                       bool prio)
{
    const int slots = phi_ctas < mu_ctas ? phi_ctas : mu_ctas;  // both sweeps cut the items alike
    cudaError_t e = launch_kp(general_phi_kernel<R, kTX, kTY, SYM, COMP>, dim3(phi_ctas), dim3(kTX * kTY),
                              general_phi_smem_bytes<R, COMP>(), s, pdl, prio, kp, (const Ph<R> *)phi, (const Mu<R> *)mu,
                             (Ph<R> *)phi_out, st, tab, tmap_in, tmap_out, splits, glist, stats, slots,
                             pdl && after_lean ? 1 : 0, (const Ph<R> *)phi_lo, (Ph<R> *)phi_out_lo);
    if (e != cudaSuccess) return e;
    return launch_kp(general_mu_kernel<R, kTX, kTY, SYM, COMP>, dim3(mu_ctas), dim3(kTX * kTY), mu_smem_bytes<R>(),
                     s, pdl, prio, kp, (const Ph<R> *)phi, (const Ph<R> *)phi_out, (const Mu<R> *)mu, (Mu<R> *)mu_out,
                     st, tab,
                    parts, splits, glist, stats, subparts, subcnt, slots, (const Mu<R> *)mu_lo, (Mu<R> *)mu_out_lo);
}

template <typename R>
cudaError_t launch_general_sweeps(const KParams<R> &kp, const void *phi, const void *mu, void *phi_out, void *mu_out,
                                  const DevState *st, const PlaneT<R> *tab, Partial *parts,
                                  const unsigned char *tmap_in, unsigned char *tmap_out, const int2 *splits,
                                  const int *glist, LeanStats *stats, int phi_ctas, int mu_ctas, cudaStream_t s,
                                  Partial *subparts, unsigned *subcnt, bool pdl, bool after_lean, const void *phi_lo,
                                  void *phi_out_lo, const void *mu_lo, void *mu_out_lo, bool prio)
{
    if (!subparts || !subcnt) return cudaErrorInvalidValue;
    const bool comp = phi_lo != nullptr;
    if (comp && (sizeof(R) != 4 || !phi_out_lo || !mu_lo || !mu_out_lo)) return cudaErrorInvalidValue;
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    if (!attr.done()) {
        cudaError_t e = general_sweep_attributes<R>();
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    if constexpr (sizeof(R) == 4) {
        if (comp)
            return launch_general_pair<R, false, true>(kp, phi, mu, phi_out, mu_out, st, tab, parts, tmap_in, tmap_out,
                                                       splits, glist, stats, phi_ctas, mu_ctas, s, subparts, subcnt,
                                                       pdl, after_lean, phi_lo, phi_out_lo, mu_lo, mu_out_lo, prio);
    }
    // the symmetric set (identity curvatures, one relaxation time) runs the instantiation compiled
    // without the general branches
    if (!kp.gen && !kp.gen_tau)
        return launch_general_pair<R, true, false>(kp, phi, mu, phi_out, mu_out, st, tab, parts, tmap_in, tmap_out,
                                                   splits, glist, stats, phi_ctas, mu_ctas, s, subparts, subcnt, pdl,
                                                   after_lean, nullptr, nullptr, nullptr, nullptr, prio);
    return launch_general_pair<R, false, false>(kp, phi, mu, phi_out, mu_out, st, tab, parts, tmap_in, tmap_out,
                                                splits, glist, stats, phi_ctas, mu_ctas, s, subparts, subcnt, pdl,
                                                after_lean, nullptr, nullptr, nullptr, nullptr, prio);
}

template <typename R>
void general_sweep_ctas_per_sm(int *phi_per_sm, int *mu_per_sm)
{
    int a = 0, b = 0;
    // the instantiation with the general branches (it needs at least the symmetric one's registers)
    if (general_sweep_attributes<R>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, general_phi_kernel<R, kTX, kTY, false>, kTX * kTY,
                                                      phi_smem_bytes<R>()) != cudaSuccess)
        a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, general_mu_kernel<R, kTX, kTY, false>, kTX * kTY,
                                                      mu_smem_bytes<R>()) != cudaSuccess)
        b = 1;
    cudaGetLastError();
    *phi_per_sm = a > 0 ? a : 1;
    *mu_per_sm = b > 0 ? b : 1;
}

template <typename R>
int general_ctas_per_sm()
{
    int n = 0;
    // the occupancy of a launch with the kernel's dynamic shared memory: its limit must be raised first
    if (cudaFuncSetAttribute(general_step_kernel<R, kTX, kTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fused_smem_bytes<R>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, general_step_kernel<R, kTX, kTY>, kTX * kTY,
                                                      fused_smem_bytes<R>()) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <typename R>
cudaError_t launch_lean_step(const KParams<R> &kp, const Geometry &g, int nsub, const void *mu_map, const void *mu,
                             void *phi_out, void *mu_out, const DevState *st, LeanStats *stats, cudaStream_t s,
                             const unsigned char *tmap_in, unsigned char *tmap_out, const int2 *splits, bool pdl,
                             const void *mu_lo, void *phi_out_lo, void *mu_out_lo)
{
    using L = LeanLayout<R, kTX, kTY>;
    // the compensated form is written for the FP32 column-pair consumers
    constexpr bool kComp = sizeof(R) == 4 && PF_LEAN_PAIRS != 0;
    const bool comp = mu_lo != nullptr;
    if (comp && (!kComp || !phi_out_lo || !mu_out_lo)) return cudaErrorInvalidValue;
    if (!mu_map || !tmap_in || !tmap_out || !splits || nsub < 1 || kp.tgx != g.gx || kp.tgy != g.gy)
        return cudaErrorInvalidValue;
    if ((kp.zchunk + nsub - 1) / nsub > kLeanMaxSub) return cudaErrorInvalidValue;  // planes per lean CTA
    if (sizeof(R) == 4 && (kp.nx & 1)) return cudaErrorInvalidValue;  // rows must be 16-byte multiples
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = L::smem_bytes(kLeanStages);
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(lean_step_kernel<R, kTX, kTY, kLeanStages, kLeanMaxSub, kLeanRows>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if constexpr (kComp)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(lean_step_kernel<R, kTX, kTY, kLeanStages, kLeanMaxSub, kLeanRows, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    dim3 grid(g.gx, g.gy, g.gz * nsub);
    if constexpr (kComp) {
        if (comp)
            return launch_k(lean_step_kernel<R, kTX, kTY, kLeanStages, kLeanMaxSub, kLeanRows, true>, grid,
                            dim3(kTX * kTY / kLeanRows + 32), sm, s, pdl, kp,
                            *reinterpret_cast<const LeanMaps *>(mu_map), (const Mu<R> *)mu, (Ph<R> *)phi_out,
                            (Mu<R> *)mu_out, st, stats, tmap_out, splits, nsub, (const Mu<R> *)mu_lo,
                            (Ph<R> *)phi_out_lo, (Mu<R> *)mu_out_lo);
    }
    return launch_k(lean_step_kernel<R, kTX, kTY, kLeanStages, kLeanMaxSub, kLeanRows>, grid,
                    dim3(kTX * kTY / kLeanRows + 32), sm, s, pdl, kp, *reinterpret_cast<const LeanMaps *>(mu_map),
                    (const Mu<R> *)mu, (Ph<R> *)phi_out, (Mu<R> *)mu_out, st, stats, tmap_out, splits, nsub,
                    (const Mu<R> *)nullptr, (Ph<R> *)nullptr, (Mu<R> *)nullptr);
}

#ifdef PF_FLOAT_UNIT
// The window decision of a decomposed domain (reading R11 on the global interface height): one thread
// sums the slabs' liquid deficits in slab order, decides the shift as finalize_body does, and applies it
// to every slab's state, so that all slabs move their rings alike.  Defined in the FP32 unit only (it
// does not depend on the stencil precision).
__global__ void split_combine_kernel(DevState *const *states, int nslabs, int nx, int ny_global, int nz, int window,
                                     double trigger)
{
    pdl_wait();
    double liq = 0.0;
    for (int q = 0; q < nslabs; q++) liq += states[q]->liq;
    const double h = liq / ((double)nx * (double)ny_global);
    int sh = 0;
    if (window && h >= trigger) {
        sh = (int)floor(h - trigger) + 1;
        if (sh > nz - 1) sh = nz - 1;
        if (sh < 0) sh = 0;
    }
    for (int q = 0; q < nslabs; q++) {
        DevState *st = states[q];
        st->h_int = h;
        st->shift = sh;
        if (sh > 0) {
            int zb = st->zbase + sh;
            if (zb >= nz) zb -= nz;
            st->zbase = zb;
            st->off = st->off + (double)sh;
            st->nshift_total += sh;
        }
    }
}
cudaError_t launch_split_combine(DevState *const *states, int nslabs, int nx, int ny_global, int nz, int window,
                                 double trigger, cudaStream_t s)
{
    split_combine_kernel<<<1, 1, 0, s>>>(states, nslabs, nx, ny_global, nz, window, trigger);
    return cudaGetLastError();
}

// compensated FP32 sweeps (the low words of the state ride along); defined in the FP32 unit only
cudaError_t launch_phi_sweep_comp(const KParams<float> &kp, const Geometry &g, const void *phi, const void *phi_lo,
                                  const void *mu, void *phi_out, void *phi_out_lo, const DevState *st,
                                  const PlaneT<float> *tab, cudaStream_t s)
{
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = phi_smem_bytes<float>() + sizeof(Ph<float>) * phi_ring<float>() * kTX * kTY;
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(phi_sweep_kernel<float, kTX, kTY, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    dim3 grid(g.gx, g.gy, g.gz);
    phi_sweep_kernel<float, kTX, kTY, true><<<grid, kTX * kTY, sm, s>>>(
        kp, (const Ph<float> *)phi, (const Mu<float> *)mu, (Ph<float> *)phi_out, st, tab, (const Ph<float> *)phi_lo,
        (Ph<float> *)phi_out_lo);
    return cudaGetLastError();
}

cudaError_t launch_mu_sweep_comp(const KParams<float> &kp, const Geometry &g, const void *phi_old,
                                 const void *phi_new, const void *mu, const void *mu_lo, void *mu_out,
                                 void *mu_out_lo, const DevState *st, const PlaneT<float> *tab, Partial *parts,
                                 cudaStream_t s)
{
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = mu_smem_bytes<float>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(mu_sweep_kernel<float, kTX, kTY, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    dim3 grid(g.gx, g.gy, g.gz);
    mu_sweep_kernel<float, kTX, kTY, true><<<grid, kTX * kTY, sm, s>>>(
        kp, (const Ph<float> *)phi_old, (const Ph<float> *)phi_new, (const Mu<float> *)mu, (Mu<float> *)mu_out, st,
        tab, parts, (const Mu<float> *)mu_lo, (Mu<float> *)mu_out_lo);
    return cudaGetLastError();
}
#endif

template <typename R>
cudaError_t launch_batched_step(const BatchDomain<R> *doms, int ndoms, const BatchItem *items, int nitems,
                                unsigned *counter, int parity, int ctas, int post_blocks, cudaStream_t s)
{
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t sm = fused_smem_bytes<R>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(batched_fused_kernel<R, kTX, kTY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    batched_fused_kernel<R, kTX, kTY><<<ctas, kTX * kTY, sm, s>>>(doms, items, nitems, counter, parity);
    batched_finalize_kernel<R><<<ndoms, 256, 0, s>>>(doms);
    batched_post_kernel<R><<<dim3(post_blocks, ndoms), 256, 0, s>>>(doms, parity);
    return cudaGetLastError();
}

// Batched step on the lean path (domains with TMA maps) and, for the other domains, the fused tile.
template <typename R>
cudaError_t launch_batched_lean_step(const BatchDomain<R> *doms, int ndoms, const int2 *plan_entries, int nplan,
                                     const int4 *lean_items, int nlean, int2 *glist, BatchPlan *plan,
                                     int phi_ctas, int mu_ctas, const BatchItem *fitems, int nfitems,
                                     unsigned *counter, int fctas, int parity, int post_blocks, cudaStream_t s,
                                     bool sym, cudaStream_t aux, cudaEvent_t fork, cudaEvent_t join, int lean_rows)
{
    using L = LeanLayout<R, kTX, kTY>;
    using LH = LeanLayout<R, kTX, kTY / 2>;
    if (lean_rows != kTY && lean_rows != kTY / 2) return cudaErrorInvalidValue;
    static DeviceOnce attr;  // the attribute is a per-device setting: set once on each device
    const size_t smp = phi_smem_bytes<R>(), smm = mu_smem_bytes<R>(), sml = L::smem_bytes(kLeanStages);
    const size_t smlh = LH::smem_bytes(kLeanStages);
    const size_t smf = fused_smem_bytes<R>();
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(batched_general_kernel<R, kTX, kTY, 0, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batched_general_kernel<R, kTX, kTY, 1, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batched_general_kernel<R, kTX, kTY, 0, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batched_general_kernel<R, kTX, kTY, 1, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smm);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batched_lean_kernel<R, kTX, kTY, kLeanStages, kLeanMaxSub, kLeanRows, kTY>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sml);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batched_lean_kernel<R, kTX, kTY / 2, kLeanStages, kLeanMaxSub, kLeanRowsHalf, kTY>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smlh);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(batched_fused_kernel<R, kTX, kTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smf);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    cudaError_t e = cudaMemsetAsync(plan, 0, sizeof(BatchPlan), s);
    if (e != cudaSuccess) return e;
    // with a second stream the general planes' sweeps run beside the lean and fused kernels (they
    // touch other planes, map entries and partials); finalize waits for both
    const bool conc = aux && fork && join && nplan > 0;
    if (nplan > 0) {
        batched_plan_kernel<R, kTX, kTY><<<(nplan + 3) / 4, 256, 0, s>>>(doms, plan_entries, nplan, parity, glist,
                                                                          plan);
        cudaStream_t g = s;
        if (conc) {
            e = cudaEventRecord(fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, fork, 0);
            if (e != cudaSuccess) return e;
            g = aux;
        }
        if (sym) {
            batched_general_kernel<R, kTX, kTY, 0, true><<<phi_ctas, kTX * kTY, smp, g>>>(doms, glist, plan, parity);
            batched_general_kernel<R, kTX, kTY, 1, true><<<mu_ctas, kTX * kTY, smm, g>>>(doms, glist, plan, parity);
        } else {
            batched_general_kernel<R, kTX, kTY, 0, false><<<phi_ctas, kTX * kTY, smp, g>>>(doms, glist, plan, parity);
            batched_general_kernel<R, kTX, kTY, 1, false><<<mu_ctas, kTX * kTY, smm, g>>>(doms, glist, plan, parity);
        }
        if (conc) {
            e = cudaEventRecord(join, aux);
            if (e != cudaSuccess) return e;
        }
    }
    if (nlean > 0 && lean_rows == kTY)
        batched_lean_kernel<R, kTX, kTY, kLeanStages, kLeanMaxSub, kLeanRows, kTY>
            <<<nlean, kTX * kTY / kLeanRows + 32, sml, s>>>(doms, lean_items, parity);
    else if (nlean > 0)
        batched_lean_kernel<R, kTX, kTY / 2, kLeanStages, kLeanMaxSub, kLeanRowsHalf, kTY>
            <<<nlean, kTX * (kTY / 2) / kLeanRowsHalf + 32, smlh, s>>>(doms, lean_items, parity);
    if (nfitems > 0) {
        e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        batched_fused_kernel<R, kTX, kTY><<<fctas, kTX * kTY, smf, s>>>(doms, fitems, nfitems, counter, parity);
    }
    if (conc) {
        e = cudaStreamWaitEvent(s, join, 0);
        if (e != cudaSuccess) return e;
    }
    batched_finalize_kernel<R><<<ndoms, 256, 0, s>>>(doms);
    batched_post_kernel<R><<<dim3(post_blocks, ndoms), 256, 0, s>>>(doms, parity);
    return cudaGetLastError();
}

template <typename R>
void batched_general_ctas_per_sm(int *phi_per_sm, int *mu_per_sm)
{
    int a = 0, b = 0;
    if (cudaFuncSetAttribute(batched_general_kernel<R, kTX, kTY, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)phi_smem_bytes<R>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, batched_general_kernel<R, kTX, kTY, 0, false>, kTX * kTY,
                                                      phi_smem_bytes<R>()) != cudaSuccess)
        a = 1;
    if (cudaFuncSetAttribute(batched_general_kernel<R, kTX, kTY, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mu_smem_bytes<R>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batched_general_kernel<R, kTX, kTY, 1, false>, kTX * kTY,
                                                      mu_smem_bytes<R>()) != cudaSuccess)
        b = 1;
    cudaGetLastError();
    *phi_per_sm = a > 0 ? a : 1;
    *mu_per_sm = b > 0 ? b : 1;
}

template <typename R>
int fused_ctas_per_sm()
{
    int n = 0;
    if (cudaFuncSetAttribute(batched_fused_kernel<R, kTX, kTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fused_smem_bytes<R>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_fused_kernel<R, kTX, kTY>, kTX * kTY,
                                                      fused_smem_bytes<R>()) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <typename R>
cudaError_t launch_finalize(const KParams<R> &kp, DevState *st, const Partial *parts, int nparts, cudaStream_t s,
                            LeanStats *lean, bool pdl)
{
    return launch_k(finalize_kernel<R>, dim3(1), dim3(256), 0, s, pdl, kp, st, parts, nparts, lean);
}

template <typename R>
cudaError_t launch_post(const KParams<R> &kp, const DevState *st, void *phi, void *mu, PlaneT<R> *tab,
                        cudaStream_t s, void *phi_lo, void *mu_lo, unsigned char *tmap, bool pdl)
{
    // enough threads to fill one full plane per thread-sweep when the window moves
    const size_t work = (size_t)kp.nx * kp.ny;
    return launch_k(post_kernel<R>, dim3(grid1d(work > (size_t)2 * kp.nz ? work : (size_t)2 * kp.nz)), dim3(256), 0,
                    s, pdl, kp, st, (Ph<R> *)phi, (Mu<R> *)mu, tab, (Ph<R> *)phi_lo, (Mu<R> *)mu_lo, tmap);
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
                          double *plane_sums, cudaStream_t s, const void *phi_lo, const void *mu_lo)
{
    reduce_kernel<R><<<kp.nz, 256, 0, s>>>(kp, st, (const Ph<R> *)phi, (const Mu<R> *)mu, plane_sums,
                                           (const Ph<R> *)phi_lo, (const Mu<R> *)mu_lo);
    return cudaGetLastError();
}

template <typename R, typename H>
cudaError_t launch_pack(const KParams<R> &kp, const DevState *st, const void *phi, const void *mu, H *phi_soa,
                        H *mu_soa, int k0, int nk, cudaStream_t s, const void *phi_lo, const void *mu_lo)
{
    const size_t n = (size_t)kp.nx * kp.ny * nk;
    pack_kernel<R, H><<<grid1d(n), 256, 0, s>>>(kp, st, (const Ph<R> *)phi, (const Mu<R> *)mu, phi_soa, mu_soa, k0,
                                                nk, (const Ph<R> *)phi_lo, (const Mu<R> *)mu_lo);
    return cudaGetLastError();
}

template <typename R, typename H>
cudaError_t launch_unpack(const KParams<R> &kp, const DevState *st, void *phi, void *mu, const H *phi_soa,
                          const H *mu_soa, int k0, int nk, cudaStream_t s, void *phi_lo, void *mu_lo)
{
    const size_t n = (size_t)kp.nx * kp.ny * nk;
    unpack_kernel<R, H><<<grid1d(n), 256, 0, s>>>(kp, st, (Ph<R> *)phi, (Mu<R> *)mu, phi_soa, mu_soa, k0, nk,
                                                  (Ph<R> *)phi_lo, (Mu<R> *)mu_lo);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mesh_count(const KParams<R> &kp, const DevState *st, const void *phi, int phase, double iso,
                              unsigned *seg_counts, cudaStream_t s)
{
    const int nb = (kp.nx + MESH_W - 1) / MESH_W;
    const unsigned gz = (unsigned)((kp.nz - 1 + MESH_KC - 1) / MESH_KC);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long wide = (long)nb * ((kp.ny + MESH_ROWS_WIDE - 1) / MESH_ROWS_WIDE) * gz;
    if (wide >= 4L * sms) {
        const dim3 grid((unsigned)(nb * ((kp.ny + MESH_ROWS_WIDE - 1) / MESH_ROWS_WIDE)), gz);
        mesh_count_kernel<R, MESH_ROWS_WIDE><<<grid, MESH_W, 0, s>>>((const Ph<R> *)phi, st, kp.nx, kp.ny, kp.nz,
                                                                     phase, (R)iso, seg_counts);
    } else {
        const dim3 grid((unsigned)(nb * ((kp.ny + MESH_ROWS_NARROW - 1) / MESH_ROWS_NARROW)), gz);
        mesh_count_kernel<R, MESH_ROWS_NARROW><<<grid, MESH_W, 0, s>>>((const Ph<R> *)phi, st, kp.nx, kp.ny, kp.nz,
                                                                       phase, (R)iso, seg_counts);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mesh_scan(const unsigned *seg_counts, size_t nseg_pad, unsigned *ne_seg, unsigned long long *ne_off,
                             unsigned long long *totals, cudaStream_t s)
{
    mesh_scan_kernel<<<1, 1024, 0, s>>>(seg_counts, nseg_pad, ne_seg, ne_off, totals);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mesh_emit(const KParams<R> &kp, const DevState *st, const void *phi, int phase, double iso,
                             const unsigned *ne_seg, const unsigned long long *ne_off, unsigned n_ne,
                             unsigned long long ntris, float *tris, cudaStream_t s)
{
    mesh_emit_kernel<R><<<n_ne, MESH_W, 0, s>>>((const Ph<R> *)phi, st, kp.nx, kp.ny, kp.nz, phase, (R)iso, ne_seg,
                                                ne_off, ntris, tris);
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
                                              cudaStream_t, const unsigned char *, unsigned char *, bool);        \
    template cudaError_t launch_classify<R>(const KParams<R> &, const DevState *, const void *, unsigned char *, \
                                            cudaStream_t, const void *);                                         \
    template cudaError_t launch_lean_step<R>(const KParams<R> &, const Geometry &, int, const void *, const void *, \
                                             void *, void *, const DevState *, LeanStats *, cudaStream_t,          \
                                             const unsigned char *, unsigned char *, const int2 *, bool,           \
                                             const void *, void *, void *);                                        \
    template cudaError_t launch_plan<R>(const KParams<R> &, const Geometry &, const DevState *,                  \
                                        const unsigned char *, int2 *, int *, LeanStats *, Partial *,            \
                                        cudaStream_t, bool);                                                     \
    template cudaError_t launch_general_step<R>(const KParams<R> &, const void *, const void *, void *, void *,  \
                                                const DevState *, const PlaneT<R> *, Partial *,                  \
                                                const unsigned char *, unsigned char *, const int2 *, const int *, \
                                                LeanStats *, int, cudaStream_t);                                 \
    template int general_ctas_per_sm<R>();                                                                       \
    template cudaError_t launch_general_sweeps<R>(const KParams<R> &, const void *, const void *, void *, void *, \
                                                  const DevState *, const PlaneT<R> *, Partial *,                  \
                                                  const unsigned char *, unsigned char *,                           \
                                                  const int2 *, const int *, LeanStats *, int, int, cudaStream_t, \
                                                  Partial *, unsigned *, bool, bool, const void *, void *,        \
                                                  const void *, void *, bool);                                     \
    template void general_sweep_ctas_per_sm<R>(int *, int *);                                                    \
    template cudaError_t launch_batched_step<R>(const BatchDomain<R> *, int, const BatchItem *, int, unsigned *, \
                                                int, int, int, cudaStream_t);                                    \
    template int fused_ctas_per_sm<R>();                                                                         \
    template cudaError_t launch_batched_lean_step<R>(const BatchDomain<R> *, int, const int2 *, int, const int4 *, \
                                                     int, int2 *, BatchPlan *, int, int, const BatchItem *, int,   \
                                                     unsigned *, int, int, int, cudaStream_t, bool, cudaStream_t, cudaEvent_t, cudaEvent_t, \
                                                     int);                                                       \
    template void batched_general_ctas_per_sm<R>(int *, int *);                                                  \
    template cudaError_t launch_finalize<R>(const KParams<R> &, DevState *, const Partial *, int, cudaStream_t,   \
                                            LeanStats *, bool);                                                  \
    template cudaError_t launch_post<R>(const KParams<R> &, const DevState *, void *, void *, PlaneT<R> *,       \
                                        cudaStream_t, void *, void *, unsigned char *, bool);                    \
    template cudaError_t launch_init<R>(const KParams<R> &, void *, void *, const double *, int, int,            \
                                        cudaStream_t);                                                           \
    template cudaError_t launch_reduce<R>(const KParams<R> &, const DevState *, const void *, const void *,      \
                                          double *, cudaStream_t, const void *, const void *);                   \
    template cudaError_t launch_pack<R, double>(const KParams<R> &, const DevState *, const void *, const void *, \
                                                double *, double *, int, int, cudaStream_t, const void *,        \
                                                const void *);                                                   \
    template cudaError_t launch_pack<R, float>(const KParams<R> &, const DevState *, const void *, const void *,  \
                                               float *, float *, int, int, cudaStream_t, const void *,           \
                                               const void *);                                                    \
    template cudaError_t launch_unpack<R, double>(const KParams<R> &, const DevState *, void *, void *,           \
                                                  const double *, const double *, int, int, cudaStream_t, void *, \
                                                  void *);                                                       \
    template cudaError_t launch_unpack<R, float>(const KParams<R> &, const DevState *, void *, void *,            \
                                                 const float *, const float *, int, int, cudaStream_t, void *,    \
                                                 void *);                                                        \
    template cudaError_t launch_mesh_count<R>(const KParams<R> &, const DevState *, const void *, int, double,    \
                                              unsigned *, cudaStream_t);                                         \
    template cudaError_t launch_mesh_scan<R>(const unsigned *, size_t, unsigned *, unsigned long long *,          \
                                             unsigned long long *, cudaStream_t);                               \
    template cudaError_t launch_mesh_emit<R>(const KParams<R> &, const DevState *, const void *, int, double,     \
                                             const unsigned *, const unsigned long long *, unsigned,            \
                                             unsigned long long, float *, cudaStream_t);

}  // namespace pf
