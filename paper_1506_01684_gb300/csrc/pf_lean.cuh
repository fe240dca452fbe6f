// pf_lean.cuh -- the pure-liquid planes of the fused step as a kernel of their own.
//
// On a lean plane (lean_split: phi^n pure liquid on the tile's 2-ring region over the planes
// q-2 .. q+2) the step reduces to the paper's liquid shortcut (Section 3.3): phi^{n+1} = e_l,
// no anti-trapping current, constant liquid mobility, so mu^{n+1} is a 7-point diffusion update
// plus the ∂c/∂T ∂T/∂t term.  The only compulsory traffic is mu^n in and mu^{n+1} out (4 words a
// cell); phi^{n+1} is stored only where the destination buffer does not already hold e_l.
//
// The kernel streams mu planes through shared memory with TMA: a producer warp issues one tensor
// copy per plane (the tile plus a one-cell halo, columns i0-2 .. i0+TX+1 so that the box starts on
// a 16-byte boundary, rows j0-1 .. j0+TY) into a ring of LD stages; at the domain's edges some
// producer lanes also store the periodic images that fall outside the tensor (the wrapped column /
// row, loaded from L2 ahead of time) into the stage; the stage's "full" mbarrier completes on the
// tensor copy's bytes and those lanes' arrivals.  TY / ROWS consumer warps wait on it, update the
// plane and release the stage through its "empty" mbarrier; a consumer thread holds ROWS cells of
// one column (FP64), or two adjacent columns of ROWS / 2 rows so that each 16-byte shared load and
// global store carries two cells (FP32).  Nothing of
// the plane sits in registers while it is in flight, so the occupancy is not bounded by the
// prefetch depth.  Every wait is bounded: a wait that gives up raises a CTA-wide abort flag, the
// producer drains the copies it issued, and the CTA reports a timeout in its partial.
#pragma once

#include <cuda.h>

#ifndef PF_LEAN_MIN_CTAS
#define PF_LEAN_MIN_CTAS 7  // resident FP32 lean CTAs per SM the register allocation must allow (FP64: 3,
                            // as many as its shared memory admits)
#endif
#ifndef PF_LEAN_SUSPEND_NS
#define PF_LEAN_SUSPEND_NS 1000u  // longest suspension of a waiting thread per try (the wait's bound is separate)
#endif

#ifndef PF_LEAN_PAIRS
#define PF_LEAN_PAIRS 1  // FP32 consumers take two adjacent columns a thread (16-byte loads and stores)
#endif
#ifndef PF_LEAN_UNROLL
#define PF_LEAN_UNROLL 1  // planes of the consumers' z-march per unrolled loop body
#endif

namespace pf {

constexpr int kLeanUnroll = PF_LEAN_UNROLL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make the barrier initialisation visible to the asynchronous (tensor copy) proxy
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// As mbar_test, but a thread whose phase is not complete is suspended until it completes or about
// hint_ns nanoseconds have passed, so a waiting warp takes no issue slots from the others.
__device__ __forceinline__ bool mbar_test_suspend(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}
// Bounded wait for the completion of the phase with the given parity.  Gives up after about 2^31
// clock cycles (about a second) and raises *abort, or as soon as another thread has raised it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test_suspend(bar, parity, PF_LEAN_SUSPEND_NS)) return true;
        if (*abort) return false;
        if (clock64() - t0 > (1LL << 31)) {
            *abort = 1;
            return false;
        }
    }
}
// tensor copy of the box at (x, y, z) of a 3D tensor map into shared memory; completes on bar
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
// barrier of the consumer warps only (the producer warp does not take part)
template <int N>
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}

// Shared-memory layout of one stage: the tensor copy of the tile box (BH rows of BW cells), then at
// 128-byte aligned offsets (a tensor copy's shared-memory destination must be 128-byte aligned) the
// boxes of the periodic images: XL the column x = nx-1 (wrapped to x = -1) and XR the column x = 0
// (wrapped to x = nx), each 2 cells x TY rows (the image is the second / first cell of each row: a
// box's first coordinate must sit on a 16-byte boundary), and YL the row y = ny-1 (wrapped to y = -1),
// YH the row y = 0 (wrapped to y = ny), each BW cells from x = i0 - 2.  Stages are 128-byte multiples
// from a 128-byte aligned base (the launch adds 128 bytes of slack for the alignment).
template <typename R, int TX, int TY>
struct LeanLayout {
    static constexpr int BW = TX + 4, BH = TY + 2, BOX = BW * BH;
    static constexpr unsigned CB = sizeof(Mu<R>);
    static constexpr unsigned up128(unsigned b) { return (b + 127u) / 128u * 128u; }
    static constexpr unsigned BOX_BYTES = BOX * CB;
    static constexpr unsigned XIMG_BYTES = 2u * TY * CB, YIMG_BYTES = BW * CB;
    static constexpr unsigned XL = up128(BOX_BYTES), XR = XL + up128(XIMG_BYTES);
    static constexpr unsigned YL = XR + up128(XIMG_BYTES), YH = YL + up128(YIMG_BYTES);
    static constexpr unsigned STAGE_BYTES = up128(YH + YIMG_BYTES);
    static constexpr size_t smem_bytes(int stages) { return (size_t)stages * STAGE_BYTES + 128; }
};

// shared-memory load of one mu cell at a byte offset (cells are 8- / 16-byte aligned)
template <typename R>
__device__ __forceinline__ Mu<R> lds_cell(const unsigned char *p)
{
    Mu<R> m;
    if constexpr (sizeof(R) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        m.v[0] = v.x;
        m.v[1] = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        m.v[0] = v.x;
        m.v[1] = v.y;
    }
    return m;
}

// Grid (tgx, tgy, gz * nsub): tile (bx, by) of the fused step's grid, z chunk blockIdx.z / nsub,
// and of that chunk the sub-chunk blockIdx.z % nsub of at most MAXSUB planes.  The CTA updates the
// chunk's lean planes (its split, from plan_kernel) that fall into its sub-chunk.  TY/ROWS consumer warps own ROWS
// consecutive tile rows each (lane = tile column), one producer warp feeds them.
// MTY: the rows of a liquid-map tile (the unit of the maps and of the plan's splits).  A CTA of TY < MTY
// rows updates the rows [by TY, by TY + TY) of map tile by / (MTY / TY) under that tile's split and
// map entries; its siblings write the same entries.  (After a timed-out wait a sibling may overwrite
// the "not known" 0 with 1; the step then latches PF_E_TIMEOUT and the maps are rebuilt when the
// fields are next initialised or written.)
// COMP: the compensated FP32 state (value = high + low word): the tensor copies carry the high words of
// mu, each consumer loads its own cells' low words, forms the increment C1 (neighbour sum - 6 mu) + C0
// from the high words and adds it to high + low with the error-free two-sum (the compensated update of
// the two sweeps); a stored pure-liquid phi gets zero low words.
template <typename R, int TX, int TY, int LD, int MAXSUB, int ROWS, bool COMP = false, int MTY = TY>
__device__ __forceinline__ void lean_tile(const KParams<R> &kp, const LeanMaps *maps, const Mu<R> *__restrict__ mu,
                                          Ph<R> *__restrict__ phi_out, Mu<R> *__restrict__ mu_out,
                                          const DevState *__restrict__ st, LeanStats *__restrict__ stats,
                                          unsigned char *__restrict__ tmap_out, const int2 *__restrict__ splits,
                                          int nsub, int bx, int by, int zsub, const Mu<R> *__restrict__ mu_lo = nullptr,
                                          Ph<R> *__restrict__ phi_out_lo = nullptr,
                                          Mu<R> *__restrict__ mu_out_lo = nullptr)
{
    using L = LeanLayout<R, TX, TY>;
    static_assert(TY % ROWS == 0, "whole rows per consumer warp");
    constexpr int NCW = TY / ROWS, NC = 32 * NCW, NTH = NC + 32;
    constexpr int CB = (int)sizeof(Mu<R>);
    constexpr bool PAIR = PF_LEAN_PAIRS != 0 && sizeof(R) == 4;
    static_assert(!COMP || PAIR, "the compensated form runs the FP32 column pairs");
    constexpr int UNR = sizeof(R) == 4 ? kLeanUnroll : 1;  // FP64 values take twice the registers
    static_assert(TX == 32 && TY % 2 == 0 && TY <= 32 && (LD & (LD - 1)) == 0, "layout");
    constexpr int LDLOG = LD == 2 ? 1 : (LD == 4 ? 2 : (LD == 8 ? 3 : 4));
    static_assert((1 << LDLOG) == LD, "LD: 2, 4, 8 or 16");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *stage_base =  // [LD][STAGE_BYTES], 128-byte aligned
        smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t full[LD], empty[LD];
    __shared__ int s_abort, s_bad;
    __shared__ unsigned char s_dst_liquid[MAXSUB];  // destination map entries of the sub-chunk's planes

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int i0 = bx * TX, j0 = by * TY;
    const int chunk = zsub / nsub, sub = zsub % nsub;
    const int z0 = chunk * kp.zchunk, z1 = min(z0 + kp.zchunk, nz);
    const int sublen = (kp.zchunk + nsub - 1) / nsub;
    const int s0 = min(z1, z0 + sub * sublen), s1 = min(z1, s0 + sublen);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;
    static_assert(MTY % TY == 0, "whole CTA tiles per map tile");
    const int ntl = kp.tgx * kp.tgy, tile = by / (MTY / TY) * kp.tgx + bx;
    auto splane = [&](int k) {
        const int sp = k + zbase;
        return sp >= nz ? sp - nz : sp;
    };
    // the periodic images this tile needs (only at the domain's edges), copied with the tile box
    const bool img_xl = bx == 0, img_xr = i0 + TX >= nx, img_yl = j0 == 0, img_yh = j0 + TY >= ny;

    // (the launch guarantees s1 - s0 <= MAXSUB) the destination's map entries, read before any is
    // replaced
    for (int q = s0 + tid; q < s1; q += NTH) s_dst_liquid[q - s0] = tmap_out[map_idx(splane(q), tile, nz)];
    if (tid == 0) {
        for (int s = 0; s < LD; s++) {
            mbar_init(&full[s], 1);    // the producer's expect-tx arrival (completion: the copies' bytes)
            mbar_init(&empty[s], NCW);  // one per consumer warp
        }
        s_abort = 0;
        s_bad = 0;
        fence_proxy_async_shared();
    }
    // the chunk's split (plan_kernel)
    const int2 sp2 = splits[(size_t)chunk * ntl + tile];
    const int lo_end = sp2.x, hi_beg = sp2.y;
    __syncthreads();  // barrier initialisation and destination map entries
    // this CTA's planes: the lean planes of the chunk that fall into its sub-chunk [s0, s1)
    int qa[2], qb[2];
    qa[0] = s0;
    qb[0] = min(s1, lo_end);
    qa[1] = max(s0, hi_beg);
    qb[1] = s1;

    if (tid >= NC) {
        // ---------------- producer warp ----------------
        const int lane = tid - NC;
        unsigned u = 0;  // stage uses issued
        bool ok = true;
        // bytes of one stage use: the tile box and the periodic images of an edge tile
        const unsigned tx_bytes = L::BOX_BYTES + (img_xl ? L::XIMG_BYTES : 0u) + (img_xr ? L::XIMG_BYTES : 0u) +
                                  (img_yl ? L::YIMG_BYTES : 0u) + (img_yh ? L::YIMG_BYTES : 0u);
        // (test hook: no copies at all, so that the consumers' bounded waits run out)
        for (int g = 0; g < 2 && ok && !(kp.test_flags & 1); g++) {
            if (qb[g] <= qa[g]) continue;
            // planes qa-1 (its mu for the z flux below qa) .. qb (for the z flux above qb-1)
            const int la = max(qa[g] - 1, 0), lb = min(qb[g], nz - 1);
            for (int p = la; p <= lb; p++, u++) {
                const int s = u & (LD - 1);
                if (u >= LD) {
                    ok = mbar_wait(&empty[s], ((u >> LDLOG) - 1) & 1, &s_abort);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                }
                unsigned char *stg = stage_base + s * L::STAGE_BYTES;
                const int sp = splane(p);
                if (lane == 0) {
                    // every copy completes on the stage's full barrier, all in the asynchronous proxy; x
                    // coordinates in words (2 a cell) sit on 16-byte boundaries (nx even in FP32)
                    mbar_arrive_expect_tx(&full[s], tx_bytes);
                    tma_load_3d(stg, &maps->box, &full[s], 2 * (i0 - 2), j0 - 1, sp);
                    if (img_xl) tma_load_3d(stg + L::XL, &maps->ximg, &full[s], 2 * (nx - 2), j0, sp);
                    if (img_xr) tma_load_3d(stg + L::XR, &maps->ximg, &full[s], 0, j0, sp);
                    if (img_yl) tma_load_3d(stg + L::YL, &maps->yimg, &full[s], 2 * (i0 - 2), ny - 1, sp);
                    if (img_yh) tma_load_3d(stg + L::YH, &maps->yimg, &full[s], 2 * (i0 - 2), 0, sp);
                }
            }
        }
        if (!ok && lane == 0) {
            // drain: the tensor copies of the last LD uses may still be landing in shared memory
            for (unsigned v = u > (unsigned)LD ? u - LD : 0; v < u; v++) {
                const long long t0 = clock64();
                while (!mbar_test(&full[v & (LD - 1)], (v >> LDLOG) & 1) && clock64() - t0 < (1LL << 31)) {
                }
            }
        }
        return;
    }

    // ---------------- consumer warps ----------------
    const int lane = tid & 31, w = tid >> 5;
    // byte offsets of the periodic images in a stage: x = -1 of tile row r at XL + (2 r + 1) CB, x = nx
    // at XR + 2 r CB, y = -1 of tile column c at YL + (c + 2) CB, y = ny at YH + (c + 2) CB
    constexpr int XL = (int)L::XL, XR = (int)L::XR, YL = (int)L::YL, YH = (int)L::YH;
    // The liquid update with constant mobility M = D_l/(2 A_l), h = e_l and no phase change (the
    // short form of Eq. 3 for a cell whose neighbourhood is pure liquid): the six face fluxes
    // M (mu_nb - mu)/dx reduce to the 7-point sum, so
    //   mu^{n+1} = mu^n + C1 (sum of the six neighbours - 6 mu^n) + C0,
    //   C1 = dt M / (chi dx^2),  C0 = -k_l dT / chi  (per component; chi = 1/(2 A_l)).
    // The zero-gradient mirror at z = 0 and z = nz-1 makes the missing neighbour the cell itself.
    // with matrix curvatures chi = K_l, M = D_l K_l: C1 = dt D_l / dx^2, C0 = -K_l^{-1} k_l dT
    // (formed on the host in FP64)
    const R ichi = rcp(kp.inv2A[3]);
    const R C1 = kp.gen ? kp.liqC1 : ichi * (kp.dt * (kp.DinvA[3] * kp.inv_dx * kp.inv_dx));
    R C0[2];
    C0[0] = kp.gen ? kp.liqC0[0] : -(kp.kT[3][0] * kp.dTstep) * ichi;
    C0[1] = kp.gen ? kp.liqC0[1] : -(kp.kT[3][1] * kp.dTstep) * ichi;
    Ph<R> liquid;
    liquid.v[0] = liquid.v[1] = liquid.v[2] = R(0);
    liquid.v[3] = R(1);
    bool ok = true;
    R acc = R(0);  // sum of the updated values: non-finite iff one of them is
    int phi_stores = 0, planes = 0;
    unsigned u = 0;  // stage uses consumed
    if constexpr (PAIR) {
        // Two adjacent columns per thread: 16-byte shared loads and global stores carry both cells'
        // mu.  Lane l holds tile columns 2 (l & 15) and 2 (l & 15) + 1 of the tile rows
        // w ROWS + (l >> 4) PR + k, k < PR; every sum is formed in the order of the one-column form.
        constexpr int PR = ROWS / 2;
        static_assert(ROWS % 2 == 0, "row pairs");
        const int c2 = lane & 15, rs = lane >> 4;
        const int ca = 2 * c2, ia = i0 + ca, ib = ia + 1;
        const int trow0 = w * ROWS + rs * PR, jr = j0 + trow0;
        const int own0 = ((trow0 + 1) * L::BW + ca + 2) * CB;
        int oxm[PR], oxp[PR], oyw[PR];
        bool vr[PR], top[PR];
#pragma unroll
        for (int k = 0; k < PR; k++) {
            const int own = own0 + k * L::BW * CB, tyr = trow0 + k, j = jr + k;
            vr[k] = ia < nx && j < ny;  // nx is even on this path: ia < nx implies ib < nx
            oxm[k] = ia == 0 ? XL + (2 * tyr + 1) * CB : own - CB;
            oxp[k] = ib == nx - 1 ? XR + 2 * tyr * CB : own + 2 * CB;
            top[k] = j == ny - 1;
            oyw[k] = top[k] ? YH + (ca + 2) * CB : own + L::BW * CB;  // the pair above row k
        }
        const int oyb = jr == 0 ? YL + (ca + 2) * CB : own0 - L::BW * CB;  // the pair below row 0
        const size_t col0 = (size_t)jr * nx + (size_t)min(ia, nx - 2);
        auto lds_pair = [](const unsigned char *p) { return *reinterpret_cast<const float4 *>(p); };
        auto lds_one = [](const unsigned char *p) { return *reinterpret_cast<const float2 *>(p); };
        for (int g = 0; g < 2 && ok; g++) {
            if (qb[g] <= qa[g]) continue;
            const int la = max(qa[g] - 1, 0), lb = min(qb[g], nz - 1);
            auto stg = [&](unsigned v) { return (const unsigned char *)stage_base + (v & (LD - 1)) * L::STAGE_BYTES; };
            auto wait_use = [&](unsigned v) {
                return __all_sync(0xffffffffu, mbar_wait(&full[v & (LD - 1)], (v >> LDLOG) & 1, &s_abort));
            };
            auto release = [&](unsigned v) {
                // the warp's shared-memory reads of the stage (generic proxy) are ordered before the
                // tensor copy that refills it (asynchronous proxy) once the producer sees this arrival;
                // without the proxy fence that copy could overwrite values still being read
                fence_proxy_async_shared();
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[v & (LD - 1)]);
            };
            unsigned v = u;
            float4 m[PR], mlo[PR];
            ok = wait_use(v);
            if (ok && qa[g] > 0) {  // plane qa - 1: only the cells below qa
#pragma unroll
                for (int k = 0; k < PR; k++) mlo[k] = lds_pair(stg(v) + own0 + k * L::BW * CB);
                release(v);
                v++;
                ok = wait_use(v);
            }
            if (ok) {
#pragma unroll
                for (int k = 0; k < PR; k++) {
                    m[k] = lds_pair(stg(v) + own0 + k * L::BW * CB);
                    if (qa[g] == 0) mlo[k] = m[k];  // mirror below plane 0
                }
            }
#pragma unroll UNR
            for (int q = qa[g]; q < qb[g] && ok; q++, v++) {
                const size_t o = (size_t)splane(q) * plane + col0;
                float4 wl[PR];  // compensated: low words of the own cells' mu^n, loaded before the waits
                if constexpr (COMP) {
#pragma unroll
                    for (int k = 0; k < PR; k++)
                        wl[k] = vr[k] ? __ldg(reinterpret_cast<const float4 *>(mu_lo + o + (size_t)k * nx))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const unsigned char *S = stg(v);
                float4 mn[PR];
#pragma unroll
                for (int k = 0; k < PR; k++) mn[k] = m[k];  // mirror above plane nz-1
                if (q < nz - 1) {
                    ok = wait_use(v + 1);
                    if (!ok) break;
                    const unsigned char *N = stg(v + 1);
#pragma unroll
                    for (int k = 0; k < PR; k++) mn[k] = lds_pair(N + own0 + k * L::BW * CB);
                }
                float2 xm[PR], xp[PR];
                float4 yhi[PR];
#pragma unroll
                for (int k = 0; k < PR; k++) {
                    xm[k] = lds_one(S + oxm[k]);
                    xp[k] = lds_one(S + oxp[k]);
                }
                const float4 ylo0 = lds_pair(S + oyb);
#pragma unroll
                for (int k = 0; k < PR; k++) {
                    if (k == PR - 1)
                        yhi[k] = lds_pair(S + oyw[k]);
                    else
                        yhi[k] = top[k] ? lds_pair(S + oyw[k]) : m[k + 1];
                }
                release(v);
                float4 out[PR], outl[PR];
#pragma unroll
                for (int k = 0; k < PR; k++) {
                    const float4 c = m[k], yl = k == 0 ? ylo0 : m[k - 1], yh = yhi[k], lo = mlo[k], hi = mn[k];
                    // cell a: x neighbours xm and cell b; cell b: cell a and xp
                    const float sa0 = ((xm[k].x + c.z) + (yl.x + yh.x)) + (lo.x + hi.x);
                    const float sa1 = ((xm[k].y + c.w) + (yl.y + yh.y)) + (lo.y + hi.y);
                    const float sb0 = ((c.x + xp[k].x) + (yl.z + yh.z)) + (lo.z + hi.z);
                    const float sb1 = ((c.y + xp[k].y) + (yl.w + yh.w)) + (lo.w + hi.w);
                    if constexpr (COMP) {
                        // The increment of a compensated state must be accurate relative to itself, not
                        // to mu: the Laplacian as a sum of neighbour differences (each exact when the
                        // values are close, as in the flux form), not as the neighbour sum minus 6 mu
                        // (whose FP32 rounding is relative to |mu|)
                        const float da0 = (((xm[k].x - c.x) + (c.z - c.x)) + ((yl.x - c.x) + (yh.x - c.x))) +
                                          ((lo.x - c.x) + (hi.x - c.x));
                        const float da1 = (((xm[k].y - c.y) + (c.w - c.y)) + ((yl.y - c.y) + (yh.y - c.y))) +
                                          ((lo.y - c.y) + (hi.y - c.y));
                        const float db0 = (((c.x - c.z) + (xp[k].x - c.z)) + ((yl.z - c.z) + (yh.z - c.z))) +
                                          ((lo.z - c.z) + (hi.z - c.z));
                        const float db1 = (((c.y - c.w) + (xp[k].y - c.w)) + ((yl.w - c.w) + (yh.w - c.w))) +
                                          ((lo.w - c.w) + (hi.w - c.w));
                        const DF r0 = df_add_f(DF{c.x, wl[k].x}, C1 * da0 + C0[0]);
                        const DF r1 = df_add_f(DF{c.y, wl[k].y}, C1 * da1 + C0[1]);
                        const DF r2 = df_add_f(DF{c.z, wl[k].z}, C1 * db0 + C0[0]);
                        const DF r3 = df_add_f(DF{c.w, wl[k].w}, C1 * db1 + C0[1]);
                        out[k] = make_float4(r0.h, r1.h, r2.h, r3.h);
                        outl[k] = make_float4(r0.l, r1.l, r2.l, r3.l);
                    } else {
                        out[k].x = C1 * (sa0 - 6.f * c.x) + (c.x + C0[0]);
                        out[k].y = C1 * (sa1 - 6.f * c.y) + (c.y + C0[1]);
                        out[k].z = C1 * (sb0 - 6.f * c.z) + (c.z + C0[0]);
                        out[k].w = C1 * (sb1 - 6.f * c.w) + (c.w + C0[1]);
                    }
                }
                const bool store_phi = s_dst_liquid[q - s0] != 1;
                phi_stores += store_phi ? 1 : 0;
                planes++;
#pragma unroll
                for (int k = 0; k < PR; k++) {
                    if (vr[k]) {
                        if (store_phi) {
                            st_ph(phi_out + o + (size_t)k * nx, liquid);
                            st_ph(phi_out + o + (size_t)k * nx + 1, liquid);
                            if constexpr (COMP) {
                                Ph<R> zero;
                                zero.v[0] = zero.v[1] = zero.v[2] = zero.v[3] = R(0);
                                st_ph(phi_out_lo + o + (size_t)k * nx, zero);
                                st_ph(phi_out_lo + o + (size_t)k * nx + 1, zero);
                            }
                        }
                        *reinterpret_cast<float4 *>(mu_out + o + (size_t)k * nx) = out[k];
                        if constexpr (COMP) *reinterpret_cast<float4 *>(mu_out_lo + o + (size_t)k * nx) = outl[k];
                        acc += (out[k].x + out[k].y) + (out[k].z + out[k].w);
                    }
                    mlo[k] = m[k];
                    m[k] = mn[k];
                }
            }
            if (ok && lb == qb[g]) release(v);  // plane qb: waited for the z neighbours of plane qb-1 only
            u += (unsigned)(lb - la + 1);
        }
    } else {
        // one column per thread: lane = tile column, warp w = tile rows w*ROWS .. w*ROWS+ROWS-1
        const int i = i0 + lane, jr0 = j0 + w * ROWS;
        // byte offsets within a stage: own cells (row r at own0 + r * BW cells), their x neighbours,
        // the cell below row 0 and the cell above each row; a neighbour across the domain edge is its
        // periodic image in the stage's wrapped-cell rows
        const int own0 = ((w * ROWS + 1) * L::BW + lane + 2) * CB;
        int oxm[ROWS], oxp[ROWS], oyu[ROWS];
        bool vr[ROWS];
    #pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const int own = own0 + r * L::BW * CB, tyr = w * ROWS + r, j = jr0 + r;
            vr[r] = i < nx && j < ny;
            oxm[r] = i == 0 ? XL + (2 * tyr + 1) * CB : own - CB;
            oxp[r] = i == nx - 1 ? XR + 2 * tyr * CB : own + CB;
            oyu[r] = j == ny - 1 ? YH + (lane + 2) * CB : own + L::BW * CB;
        }
        const int oyb = jr0 == 0 ? YL + (lane + 2) * CB : own0 - L::BW * CB;
        const size_t col0 = (size_t)jr0 * nx + (size_t)min(i, nx - 1);
        for (int g = 0; g < 2 && ok; g++) {
            if (qb[g] <= qa[g]) continue;
            const int la = max(qa[g] - 1, 0), lb = min(qb[g], nz - 1);
            // use v holds plane la + (v - u): stage v mod LD, phase parity (v / LD) mod 2
            auto stg = [&](unsigned v) { return (const unsigned char *)stage_base + (v & (LD - 1)) * L::STAGE_BYTES; };
            auto wait_use = [&](unsigned v) {
                return __all_sync(0xffffffffu, mbar_wait(&full[v & (LD - 1)], (v >> LDLOG) & 1, &s_abort));
            };
            auto release = [&](unsigned v) {
                // the warp's shared-memory reads of the stage (generic proxy) are ordered before the
                // tensor copy that refills it (asynchronous proxy) once the producer sees this arrival;
                // without the proxy fence that copy could overwrite values still being read
                fence_proxy_async_shared();
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[v & (LD - 1)]);
            };
            unsigned v = u;  // use of the plane being updated
            Mu<R> m[ROWS], mlo[ROWS];  // mu^n of the cells and of the cells below them
            ok = wait_use(v);
            if (ok && qa[g] > 0) {  // plane qa - 1: only the cells below qa
    #pragma unroll
                for (int r = 0; r < ROWS; r++) mlo[r] = lds_cell<R>(stg(v) + own0 + r * L::BW * CB);
                release(v);
                v++;
                ok = wait_use(v);
            }
            if (ok) {
    #pragma unroll
                for (int r = 0; r < ROWS; r++) {
                    m[r] = lds_cell<R>(stg(v) + own0 + r * L::BW * CB);
                    if (qa[g] == 0) mlo[r] = m[r];  // mirror below plane 0
                }
            }
    #pragma unroll UNR
            for (int q = qa[g]; q < qb[g] && ok; q++, v++) {
                const unsigned char *S = stg(v);
                Mu<R> mn[ROWS];
    #pragma unroll
                for (int r = 0; r < ROWS; r++) mn[r] = m[r];  // mirror above plane nz-1
                if (q < nz - 1) {
                    ok = wait_use(v + 1);
                    if (!ok) break;
                    const unsigned char *N = stg(v + 1);
    #pragma unroll
                    for (int r = 0; r < ROWS; r++) mn[r] = lds_cell<R>(N + own0 + r * L::BW * CB);
                }
                Mu<R> xm[ROWS], xp[ROWS];
    #pragma unroll
                for (int r = 0; r < ROWS; r++) {
                    xm[r] = lds_cell<R>(S + oxm[r]);
                    xp[r] = lds_cell<R>(S + oxp[r]);
                }
                // y neighbours: the rows of this thread, the cell below row 0 and above row ROWS-1 (or
                // their periodic images); a last domain row's upper neighbour is its periodic image
                Mu<R> yd[ROWS + 1];
                yd[0] = lds_cell<R>(S + oyb);
    #pragma unroll
                for (int r = 1; r < ROWS; r++) yd[r] = m[r];
                yd[ROWS] = lds_cell<R>(S + oyu[ROWS - 1]);
                Mu<R> wrap_up[ROWS];
    #pragma unroll
                for (int r = 0; r < ROWS - 1; r++)
                    if (jr0 + r == ny - 1) wrap_up[r] = lds_cell<R>(S + oyu[r]);
                release(v);
                Mu<R> out[ROWS];
    #pragma unroll
                for (int r = 0; r < ROWS; r++) {
                    const Mu<R> ylo = r == 0 ? yd[0] : m[r - 1];
                    const Mu<R> yhi = (r < ROWS - 1 && jr0 + r == ny - 1) ? wrap_up[r] : yd[r + 1];
    #pragma unroll
                    for (int c = 0; c < 2; c++) {
                        const R sum = ((xm[r].v[c] + xp[r].v[c]) + (ylo.v[c] + yhi.v[c])) + (mlo[r].v[c] + mn[r].v[c]);
                        const R lap = sum - R(6) * m[r].v[c];
                        out[r].v[c] = C1 * lap + (m[r].v[c] + C0[c]);
                    }
                }
                const bool store_phi = s_dst_liquid[q - s0] != 1;
                phi_stores += store_phi ? 1 : 0;
                planes++;
                const size_t o = (size_t)splane(q) * plane + col0;
    #pragma unroll
                for (int r = 0; r < ROWS; r++) {
                    if (vr[r]) {
                        if (store_phi) st_ph(phi_out + o + (size_t)r * nx, liquid);
                        st_mu(mu_out + o + (size_t)r * nx, out[r]);
                        acc += out[r].v[0] + out[r].v[1];
                    }
                    mlo[r] = m[r];
                    m[r] = mn[r];
                }
            }
            if (ok && lb == qb[g]) release(v);  // plane qb: waited for the z neighbours of plane qb-1 only
            u += (unsigned)(lb - la + 1);
        }
    }
    const bool bad = !isfinite(acc);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&s_bad, 1);
    consumer_sync<NC>();  // every consumer warp has posted its flags
    // the new field's map entries of the lean planes: pure liquid (the old entries were read at the
    // start).  After a timeout the planes' content is not known: 0, "not known to be pure liquid",
    // is always a safe entry.
    const unsigned char mark = s_abort ? 0 : 1;
    for (int g = 0; g < 2; g++)
        for (int q = qa[g] + tid; q < qb[g]; q += NC) tmap_out[map_idx(splane(q), tile, nz)] = mark;
    if (tid == 0) {
        const unsigned long long tile_cells = (unsigned long long)min(TX, nx - i0) * (unsigned long long)min(TY, ny - j0);
        // mu^n in, mu^{n+1} out (4 words a cell), plus phi^{n+1} where it was stored
        // (the compensated state moves the low words too: twice the words)
        const unsigned long long b =
            tile_cells * sizeof(R) * (COMP ? 8ull : 4ull) * (unsigned long long)(planes + phi_stores);
        if (b) atomicAdd(&stats->bytes, b);
        if (s_bad) atomicOr(&stats->nonfinite, 1);
        if (s_abort) {
            atomicOr(&stats->timeout, 1);
            atomicOr(&stats->map_changed, 1);  // its planes' map entries were set to 0 ("not known")
        }
    }
}

// The lean planes of one domain: grid (tgx, tgy, gz * nsub).  COMP: the compensated FP32 state (the low
// words of mu in and out, of phi out).
template <typename R, int TX, int TY, int LD, int MAXSUB, int ROWS, bool COMP = false>
__global__ void __launch_bounds__(TX *TY / ROWS + 32, sizeof(R) == 4 ? PF_LEAN_MIN_CTAS : 3) lean_step_kernel(
    const KParams<R> kp, const __grid_constant__ LeanMaps mu_map, const Mu<R> *__restrict__ mu,
    Ph<R> *__restrict__ phi_out, Mu<R> *__restrict__ mu_out, const DevState *__restrict__ st,
    LeanStats *__restrict__ stats, unsigned char *__restrict__ tmap_out, const int2 *__restrict__ splits, int nsub,
    const Mu<R> *__restrict__ mu_lo, Ph<R> *__restrict__ phi_out_lo, Mu<R> *__restrict__ mu_out_lo)
{
    pdl_wait();  // the step's plan; every CTA has passed it before the kernel behind may be scheduled
    pdl_trigger();
    lean_tile<R, TX, TY, LD, MAXSUB, ROWS, COMP>(kp, &mu_map, mu, phi_out, mu_out, st, stats, tmap_out, splits, nsub,
                                                 blockIdx.x, blockIdx.y, blockIdx.z, mu_lo, phi_out_lo, mu_out_lo);
}

// One lean work item of a batched step: CTA blockIdx.x takes (domain, tile x, TY-row block y, chunk *
// nsub + sub) from the table; the domain's tensor maps (boxes of TY + 2 rows) live in device memory
// (64-byte aligned).  MTY: the rows of a liquid-map tile.
template <typename R, int TX, int TY, int LD, int MAXSUB, int ROWS, int MTY>
__global__ void __launch_bounds__(TX *TY / ROWS + 32, sizeof(R) == 4 ? PF_LEAN_MIN_CTAS : 3) batched_lean_kernel(
    const BatchDomain<R> *__restrict__ doms, const int4 *__restrict__ items, int parity)
{
    const int4 w = items[blockIdx.x];
    const BatchDomain<R> *d = doms + w.x;
    const int a = parity, b = parity ^ 1;
    lean_tile<R, TX, TY, LD, MAXSUB, ROWS, false, MTY>(d->kp, d->mu_map + a, (const Mu<R> *)d->mu[a], (Ph<R> *)d->phi[b],
                                           (Mu<R> *)d->mu[b], d->st, d->lean, d->tmap[b], d->splits, d->nsub, w.y,
                                           w.z, w.w);
}

}  // namespace pf
