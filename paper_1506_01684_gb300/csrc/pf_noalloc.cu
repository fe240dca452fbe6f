// pf_noalloc.cu -- the allocation-free step entry point (include/pf.h, pf_step_noalloc).
//
// All scratch of one step lives in g_scratch, a file-scope device array: the step state, the
// per-plane temperature table and the per-CTA partial sums of the mu-sweep.  Host code must not
// hand g_scratch itself to a kernel: in host code that name is a host-side stand-in, not a
// device address.  The device address is looked up once per device with cudaGetSymbolAddress
// (with that device current) and cached.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "pf_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[PF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device (set-up on the first call per device).
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PF_E_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return PF_E_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return PF_OK;
}

// Sets the step state from the call's arguments (no host buffer involved), clearing the
// fields that must start at zero.
__global__ void noalloc_state_kernel(pf::DevState *st, double t, double off)
{
    st->t = t;
    st->off = off;
    st->h_int = 0.0;
    st->zbase = 0;
    st->shift = 0;
    st->nonfinite = 0;
    st->nshift_total = 0;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// The scratch layout the header documents: a 256-byte slot for the step state, 32 bytes per CTA partial.
static_assert(sizeof(pf::DevState) <= 256, "the step state fits its 256-byte slot");
static_assert(sizeof(pf::Partial) == 32, "one partial-sum record is 32 bytes");
static_assert(sizeof(pf::PlaneT<float>) == 16 * 4 && sizeof(pf::PlaneT<double>) == 16 * 8, "16-word plane entries");

template <typename R>
int noalloc_step(int nx, int ny, int nz, const pf_params &p, double t, double off, const void *phi_src,
                 const void *mu_src, void *phi_dst, void *mu_dst, double *h_int_out, cudaStream_t s)
{
    const pf::Geometry g = pf::make_geometry(nx, ny, nz, 0);
    const size_t state_b = 256;
    const size_t tab_b = round256((size_t)2 * nz * sizeof(pf::PlaneT<R>));
    const size_t part_b = (size_t)g.nparts() * sizeof(pf::Partial);
    if (state_b + tab_b + part_b > (size_t)PF_NOALLOC_SCRATCH_BYTES) return PF_E_INVAL;
    void *base = nullptr;
    int r = scratch_address(&base);
    if (r != PF_OK) return r;
    unsigned char *b = (unsigned char *)base;
    pf::DevState *st = (pf::DevState *)b;
    pf::PlaneT<R> *tab = (pf::PlaneT<R> *)(b + state_b);
    pf::Partial *parts = (pf::Partial *)(b + state_b + tab_b);

    pf_params q = p;
    q.dt = pf::resolved_dt(p, nz);
    q.window_trigger_z = 0.0;  // this call never moves the window
    const pf::KParams<R> kp = pf::kparams_for<R>(q, nx, ny, nz, g);

    noalloc_state_kernel<<<1, 1, 0, s>>>(st, t, off);
    cudaError_t e = cudaGetLastError();
    // plane table for (t, off); with shift = 0 the post kernel fills nothing
    if (e == cudaSuccess) e = pf::launch_post<R>(kp, st, (void *)phi_src, (void *)mu_src, tab, s);
    if (e == cudaSuccess) e = pf::launch_phi_sweep<R>(kp, g, phi_src, mu_src, phi_dst, st, tab, s);
    if (e == cudaSuccess) e = pf::launch_mu_sweep<R>(kp, g, phi_src, phi_dst, mu_src, mu_dst, st, tab, parts, s);
    if (e == cudaSuccess) e = pf::launch_finalize<R>(kp, st, parts, g.nparts(), s);
    if (e != cudaSuccess) return PF_E_CUDA;
    if (h_int_out) {
        pf::DevState ds;
        e = cudaMemcpyAsync(&ds, st, sizeof ds, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return PF_E_CUDA;
        *h_int_out = ds.h_int;
        if (ds.nonfinite) return PF_E_UNSTABLE;
    }
    return PF_OK;
}

}  // namespace

extern "C" int pf_step_noalloc(int nx, int ny, int nz, const pf_params *p, double t, double window_offset,
                               const void *phi_src, const void *mu_src, void *phi_dst, void *mu_dst,
                               double *h_int_out, void *stream)
{
    if (!p || !phi_src || !mu_src || !phi_dst || !mu_dst) return PF_E_INVAL;
    if (nx < 1 || ny < 1 || nz < 1) return PF_E_INVAL;
    if ((size_t)nx * ny > (size_t)1 << 31 || (size_t)nz > (size_t)1 << 24) return PF_E_INVAL;
    if (pf::validate_params(p) != PF_OK) return PF_E_INVAL;
    const uintptr_t mu_align = p->precision == PF_FP64 ? 16 : 8;
    if (((uintptr_t)phi_src | (uintptr_t)phi_dst) % 16 != 0) return PF_E_INVAL;
    if (((uintptr_t)mu_src | (uintptr_t)mu_dst) % mu_align != 0) return PF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->precision == PF_FP64)
        return noalloc_step<double>(nx, ny, nz, *p, t, window_offset, phi_src, mu_src, phi_dst, mu_dst, h_int_out, s);
    if (p->precision == PF_FP32)
        return noalloc_step<float>(nx, ny, nz, *p, t, window_offset, phi_src, mu_src, phi_dst, mu_dst, h_int_out, s);
    return PF_E_INVAL;
}
