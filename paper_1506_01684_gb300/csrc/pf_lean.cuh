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
// a 16-byte boundary, rows j0-1 .. j0+TY) into a ring of LD stages, plus asynchronous copies of
// the periodic images that fall outside the tensor (the wrapped column / row at the domain edge);
// both complete on the stage's "full" mbarrier.  Eight consumer warps (one thread per column)
// wait on it, update the plane, and release the stage through its "empty" mbarrier.  Nothing of
// the plane sits in registers while it is in flight, so the occupancy is not bounded by the
// prefetch depth.  Every wait is bounded: a wait that gives up raises a CTA-wide abort flag, the
// producer drains the copies it issued, and the CTA reports a timeout in its partial.
#pragma once

#include <cuda.h>

namespace pf {

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
// Bounded wait for the completion of the phase with the given parity.  Gives up after about 2^31
// clock cycles (about a second) and raises *abort, or as soon as another thread has raised it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
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
// asynchronous copy of B bytes (one mu cell) from global to shared memory
template <int B>
__device__ __forceinline__ void cp_async_bytes(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(B) : "memory");
}
// one expected arrival on bar, made once this thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// barrier of the consumer warps only (the producer warp does not take part)
template <int N>
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}

// Shared-memory layout of one stage: the TMA box (BH rows of BW cells) and four 32-cell rows of
// wrapped halo cells: x = -1 (-> nx-1) per tile row, x = nx (-> 0) per tile row, y = -1
// (-> ny-1) per tile column, y = ny (-> 0) per tile column.  A tensor copy's shared-memory
// destination must be 128-byte aligned: stages are 128-byte multiples from a 128-byte aligned base
// (the launch adds 128 bytes of slack for the alignment).
template <typename R, int TX, int TY>
struct LeanLayout {
    static constexpr int BW = TX + 4, BH = TY + 2, BOX = BW * BH, FIX = 4 * 32;
    static constexpr unsigned BOX_BYTES = BOX * sizeof(Mu<R>);
    static constexpr unsigned STAGE_BYTES = ((BOX + FIX) * sizeof(Mu<R>) + 127) / 128 * 128;
    static constexpr size_t smem_bytes(int stages) { return (size_t)stages * STAGE_BYTES + 128; }
};

template <typename R, int TX, int TY, int LD>
__global__ void __launch_bounds__(TX *TY + 32) lean_step_kernel(
    const KParams<R> kp, const __grid_constant__ CUtensorMap mu_map, const Mu<R> *__restrict__ mu,
    Ph<R> *__restrict__ phi_out, Mu<R> *__restrict__ mu_out, const DevState *__restrict__ st,
    const PlaneT<R> *__restrict__ tab, Partial *__restrict__ parts, const unsigned char *__restrict__ tmap_in,
    unsigned char *__restrict__ tmap_out, int nsub)
{
    using L = LeanLayout<R, TX, TY>;
    constexpr int NC = TX * TY, NTH = NC + 32;
    static_assert(TX == 32 && TY <= 32, "one warp per tile row; halo rows fit a warp");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *stage_base =  // [LD][STAGE_BYTES], 128-byte aligned
        smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t full[LD], empty[LD];
    __shared__ int kred[NTH / 32][2];
    __shared__ int s_abort, s_bad;

    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    const int tid = threadIdx.x;
    const int bx = blockIdx.x, by = blockIdx.y;
    const int i0 = bx * TX, j0 = by * TY;
    const int chunk = blockIdx.z / nsub, sub = blockIdx.z % nsub;
    const int z0 = chunk * kp.zchunk, z1 = min(z0 + kp.zchunk, nz);
    const int sublen = (kp.zchunk + nsub - 1) / nsub;
    const int s0 = min(z1, z0 + sub * sublen), s1 = min(z1, s0 + sublen);
    const int zbase = st->zbase;
    const size_t plane = (size_t)nx * ny;
    const int ntl = kp.tgx * kp.tgy, tile = by * kp.tgx + bx;
    auto splane = [&](int k) {
        const int sp = k + zbase;
        return sp >= nz ? sp - nz : sp;
    };

    if (tid == 0) {
        for (int s = 0; s < LD; s++) {
            mbar_init(&full[s], 1 + 32);  // the producer's expect-tx arrival + one per producer lane
            mbar_init(&empty[s], TY);     // one per consumer warp
        }
        s_abort = 0;
        s_bad = 0;
        fence_proxy_async_shared();
    }
    // (lean_split's barrier publishes the initialisation)
    int lo_end, hi_beg;
    lean_split<TX, TY, NTH>(tmap_in, kp.tgx, kp.tgy, nx, ny, nz, zbase, bx, by, z0, z1, kred, lo_end, hi_beg);
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
        for (int g = 0; g < 2 && ok; g++) {
            if (qb[g] <= qa[g]) continue;
            // planes qa-1 (its mu for the z flux below qa) .. qb (for the z flux above qb-1)
            const int la = max(qa[g] - 1, 0), lb = min(qb[g], nz - 1);
            for (int p = la; p <= lb; p++, u++) {
                const int s = u % LD;
                if (u >= LD) {
                    ok = mbar_wait(&empty[s], ((u / LD) - 1) & 1, &s_abort);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                }
                Mu<R> *stg = reinterpret_cast<Mu<R> *>(stage_base + s * L::STAGE_BYTES);
                const int sp = splane(p);
                if (lane == 0) {
                    mbar_arrive_expect_tx(&full[s], L::BOX_BYTES);
                    tma_load_3d(stg, &mu_map, &full[s], 2 * (i0 - 2), j0 - 1, sp);
                }
                const Mu<R> *mp = mu + (size_t)sp * plane;
                Mu<R> *fix = stg + L::BOX;
                if (bx == 0 && lane < TY && j0 + lane < ny)
                    cp_async_bytes<sizeof(Mu<R>)>(fix + lane, mp + (size_t)(j0 + lane) * nx + (nx - 1));
                if (i0 + TX >= nx && lane < TY && j0 + lane < ny)
                    cp_async_bytes<sizeof(Mu<R>)>(fix + 32 + lane, mp + (size_t)(j0 + lane) * nx);
                if (by == 0 && i0 + lane < nx)
                    cp_async_bytes<sizeof(Mu<R>)>(fix + 64 + lane, mp + (size_t)(ny - 1) * nx + i0 + lane);
                if (j0 + TY >= ny && i0 + lane < nx) cp_async_bytes<sizeof(Mu<R>)>(fix + 96 + lane, mp + i0 + lane);
                cp_async_arrive_noinc(&full[s]);
            }
        }
        cp_async_wait_all();
        if (!ok && lane == 0) {
            // drain: the tensor copies of the last LD uses may still be landing in shared memory
            for (unsigned v = u > (unsigned)LD ? u - LD : 0; v < u; v++) {
                const long long t0 = clock64();
                while (!mbar_test(&full[v % LD], (v / LD) & 1) && clock64() - t0 < (1LL << 31)) {
                }
            }
        }
        return;
    }

    // ---------------- consumer warps: thread (tx, ty) owns column (i0 + tx, j0 + ty) ----------------
    const int tx = tid % TX, ty = tid / TX, lane = tid & 31;
    const int i = i0 + tx, j = j0 + ty;
    const bool valid = i < nx && j < ny;
    const size_t col = valid ? (size_t)j * nx + i : 0;
    const int own = (ty + 1) * L::BW + tx + 2;
    Ph<R> liquid;
    liquid.v[0] = liquid.v[1] = liquid.v[2] = R(0);
    liquid.v[3] = R(1);
    bool bad = false, ok = true;
    int phi_stores = 0, planes = 0;
    unsigned u = 0;  // stage uses consumed
    for (int g = 0; g < 2 && ok; g++) {
        if (qb[g] <= qa[g]) continue;
        const int la = max(qa[g] - 1, 0), lb = min(qb[g], nz - 1);
        const unsigned ub = u;
        auto stg = [&](int p) {
            return reinterpret_cast<const Mu<R> *>(stage_base + ((ub + (unsigned)(p - la)) % LD) * L::STAGE_BYTES);
        };
        auto wait_plane = [&](int p) {
            const unsigned v = ub + (unsigned)(p - la);
            return __all_sync(0xffffffffu, mbar_wait(&full[v % LD], (v / LD) & 1, &s_abort));
        };
        auto release = [&](int p) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[(ub + (unsigned)(p - la)) % LD]);
        };
        Mu<R> Vz_lo;
        Vz_lo.v[0] = Vz_lo.v[1] = R(0);
        ok = wait_plane(la);
        if (ok && qa[g] > 0) {  // la = qa - 1: only the z flux below qa
            ok = wait_plane(qa[g]);
            if (ok) {
                Vz_lo = quiet_zflux(kp, stg(la)[own], stg(qa[g])[own]);
                release(la);
            }
        }
        for (int q = qa[g]; q < qb[g] && ok; q++) {
            const Mu<R> *B = stg(q);
            const Mu<R> *F = B + L::BOX;
            const Mu<R> mP = B[own];
            Mu<R> Vz_hi;
            Vz_hi.v[0] = Vz_hi.v[1] = R(0);
            if (q < nz - 1) {
                ok = wait_plane(q + 1);
                if (!ok) break;
                Vz_hi = quiet_zflux(kp, mP, stg(q + 1)[own]);
            }
            const Mu<R> xm = i == 0 ? F[ty] : B[own - 1];
            const Mu<R> xp = i == nx - 1 ? F[32 + ty] : B[own + 1];
            const Mu<R> ym = j == 0 ? F[64 + tx] : B[own - L::BW];
            const Mu<R> yp = j == ny - 1 ? F[96 + tx] : B[own + L::BW];
            const Mu<R> out = quiet_mu_cell(kp, tab + q, mP, xm, xp, ym, yp, Vz_lo, Vz_hi);
            release(q);
            const int sp = splane(q);
            const bool store_phi = tmap_out[(size_t)sp * ntl + tile] != 1;
            phi_stores += store_phi ? 1 : 0;
            planes++;
            if (valid) {
                if (store_phi) st_ph(phi_out + (size_t)sp * plane + col, liquid);
                st_mu(mu_out + (size_t)sp * plane + col, out);
                bad = bad | !isfinite(out.v[0] + out.v[1]);
            }
            Vz_lo = Vz_hi;
        }
        if (ok && lb == qb[g]) release(lb);  // waited for the z flux of plane qb-1, not updated here
        u = ub + (unsigned)(lb - la + 1);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&s_bad, 1);
    // every consumer has read the destination's map entries before any is replaced by the new
    // field's (the lean planes of the new field are pure liquid)
    consumer_sync<NC>();
    // (after a timeout the planes' content is not known: 0, "not known to be pure liquid", is
    // always a safe entry)
    const unsigned char mark = s_abort ? 0 : 1;
    for (int g = 0; g < 2; g++)
        for (int q = qa[g] + tid; q < qb[g]; q += NC) tmap_out[(size_t)splane(q) * ntl + tile] = mark;
    if (tid == 0) {
        Partial *part = parts + ((size_t)blockIdx.z * gridDim.y + by) * gridDim.x + bx;
        const double tile_cells = (double)min(TX, nx - i0) * (double)min(TY, ny - j0);
        part->liq_deficit = 0.0;
        part->nonfinite = s_bad ? 1.0 : 0.0;
        // mu^n in, mu^{n+1} out (4 words a cell), plus phi^{n+1} where it was stored
        part->bytes = tile_cells * (double)sizeof(R) * 4.0 * (double)(planes + phi_stores);
        part->timeout = s_abort ? 1.0 : 0.0;
    }
}

}  // namespace pf
