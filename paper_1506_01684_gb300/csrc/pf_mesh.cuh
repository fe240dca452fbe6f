// pf_mesh.cuh -- per-phase interface meshes (the paper's isosurface output of each phase,
// Section 3.2): the isosurface phi_a = iso of the current field by marching tetrahedra over the
// grid of cell centres.
//
// A cube has the cell centres (i + a, j + b, k + c), a, b, c in {0, 1}, as corners (corner n = a +
// 2b + 4c), wraps periodically in x and y (the position of column nx stays nx) and not in z:
// nx * ny * (nz - 1) cubes in the order c = (k ny + j) nx + i.  Each cube is cut into the six
// tetrahedra of its Kuhn triangulation (corner 0, then the three axes added in the order of a
// permutation, permutations in lexicographic order), which cut shared faces alike, so the surface
// has no cracks.  A corner is inside when its value is >= iso.  One inside (or outside) corner: one
// triangle through the edges from that corner to the other three (in increasing corner order); two
// inside corners a < b and outside c < d: the triangles (ac, ad, bd) and (ac, bd, bc).  A vertex on
// an edge from inside corner p to outside corner q is p + t (q - p), t = (iso - f_p) / (f_q - f_p).
// The normal (v1 - v0) x (v2 - v0) of a triangle points from the tetrahedron's inside corners to its
// outside ones (else v1 and v2 are swapped).  Classification, t and the orientation use the field's
// precision, the orientation in coordinates local to the cube (exact corner offsets 0 / 1, so that
// the sign does not depend on how far the cube is from the origin); a position is the cube's base
// (exact) plus the local vertex, rounded to FP32.  Triangles are written in the order cube,
// tetrahedron, triangle.
#pragma once

namespace pf {

__device__ __forceinline__ void kuhn_tet(int q, int (&v)[4])
{
    // permutations of (x, y, z) in lexicographic order: 012 021 102 120 201 210
    const int ax[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int pos = 0;
    v[0] = 0;
#pragma unroll
    for (int s = 0; s < 3; s++) {
        pos |= 1 << ax[q][s];
        v[s + 1] = pos;
    }
}

template <typename R>
__device__ __forceinline__ int tet_count(const R (&f)[8], int q, R iso)
{
    int v[4];
    kuhn_tet(q, v);
    int n = 0;
#pragma unroll
    for (int s = 0; s < 4; s++) n += f[v[s]] >= iso ? 1 : 0;
    return n == 0 || n == 4 ? 0 : (n == 2 ? 2 : 1);
}

template <typename R>
__device__ __forceinline__ void corner_values(const Ph<R> *__restrict__ phi, int nx, int ny, int nz, int zbase,
                                              int phase, int i, int j, int k, R (&f)[8])
{
    const size_t plane = (size_t)nx * ny;
    const int i1 = i + 1 == nx ? 0 : i + 1, j1 = j + 1 == ny ? 0 : j + 1;
#pragma unroll
    for (int n = 0; n < 8; n++) {
        const int ii = (n & 1) ? i1 : i, jj = (n & 2) ? j1 : j, kk = k + ((n >> 2) & 1);
        f[n] = phi[plane_off(kk, nz, zbase, plane) + (size_t)jj * nx + ii].v[phase];
    }
}

template <typename R>
__device__ __forceinline__ int cube_count(const R (&f)[8], R iso)
{
    int t = 0;
#pragma unroll
    for (int q = 0; q < 6; q++) t += tet_count(f, q, iso);
    return t;
}

// the triangles of tetrahedron q of a cube (corner values f, base position bx, by, bz) at out
// (9 floats each); returns how many
template <typename R>
__device__ __forceinline__ int tet_emit(const R (&f)[8], int q, R iso, R bx, R by, R bz, float *__restrict__ out)
{
    int v[4];
    kuhn_tet(q, v);
    int in[4], ou[4], ni = 0, no = 0;
#pragma unroll
    for (int s = 0; s < 4; s++) {
        if (f[v[s]] >= iso)
            in[ni++] = v[s];
        else
            ou[no++] = v[s];
    }
    if (ni == 0 || ni == 4) return 0;
    // local vertex on the edge from inside corner a to outside corner b
    auto vert = [&](int a, int b, R (&p)[3]) {
        const R t = (iso - f[a]) / (f[b] - f[a]);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const R ca = (R)((a >> d) & 1), cb = (R)((b >> d) & 1);
            p[d] = ca + t * (cb - ca);
        }
    };
    R tri[2][3][3];
    int nt;
    if (ni == 1) {
        for (int s = 0; s < 3; s++) vert(in[0], ou[s], tri[0][s]);
        nt = 1;
    } else if (ni == 3) {
        for (int s = 0; s < 3; s++) vert(in[s], ou[0], tri[0][s]);
        nt = 1;
    } else {
        R ac[3], ad[3], bd[3], bc[3];
        vert(in[0], ou[0], ac);
        vert(in[0], ou[1], ad);
        vert(in[1], ou[1], bd);
        vert(in[1], ou[0], bc);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            tri[0][0][d] = ac[d];
            tri[0][1][d] = ad[d];
            tri[0][2][d] = bd[d];
            tri[1][0][d] = ac[d];
            tri[1][1][d] = bd[d];
            tri[1][2][d] = bc[d];
        }
        nt = 2;
    }
    // inside -> outside direction of the tetrahedron (means of the local corner positions)
    R dir[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        R si = 0, so = 0;
        for (int s = 0; s < ni; s++) si += (R)((in[s] >> d) & 1);
        for (int s = 0; s < no; s++) so += (R)((ou[s] >> d) & 1);
        dir[d] = so / (R)no - si / (R)ni;
    }
    const R base[3] = {bx, by, bz};
    for (int m = 0; m < nt; m++) {
        R e1[3], e2[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            e1[d] = tri[m][1][d] - tri[m][0][d];
            e2[d] = tri[m][2][d] - tri[m][0][d];
        }
        const R n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2],
                n2 = e1[0] * e2[1] - e1[1] * e2[0];
        const bool flip = n0 * dir[0] + n1 * dir[1] + n2 * dir[2] < (R)0;
        float *o = out + 9 * m;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            o[d] = (float)(base[d] + tri[m][0][d]);
            o[3 + d] = (float)(base[d] + tri[m][flip ? 2 : 1][d]);
            o[6 + d] = (float)(base[d] + tri[m][flip ? 1 : 2][d]);
        }
    }
    return nt;
}

// The cubes are counted and emitted in segments: segment (k, j, b) holds the cubes i = 256 b ..
// 256 b + 255 (< nx) of row j of layer k, so that segments in the order (k ny + j) nb + b keep the
// cube order.  Pass 1 counts the triangles of each segment (a CTA marches MESH_KC layers of one
// row piece, one thread per cube, the x + 1 corners taken from the next lane); pass 2 (one CTA)
// scans the counts into the offsets of the segments that have triangles and lists them; pass 3
// writes the triangles of the listed segments.
constexpr int MESH_W = 256;  // cubes of a row per segment (one thread each; one mask-table entry each)
#ifndef PF_MESH_KC
#define PF_MESH_KC 32
#endif
constexpr int MESH_KC = PF_MESH_KC;        // layers per counting CTA

// Triangles of a cube from its inside mask (bit n set when corner n is inside): the tetrahedron
// rule of tet_count on the mask's bits.
__device__ __forceinline__ int mask_count(int m)
{
    int t = 0;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        int v[4];
        kuhn_tet(q, v);
        int n = 0;
#pragma unroll
        for (int s = 0; s < 4; s++) n += (m >> v[s]) & 1;
        t += n == 0 || n == 4 ? 0 : (n == 2 ? 2 : 1);
    }
    return t;
}

// Cube rows a counting CTA marches together: 8 where that still gives the launch at least 4 CTAs an
// SM, else 2 (256x256x1024: 8 rows 0.90, 4 rows 0.88, 2 rows 0.89 of the measured HBM copy rate;
// 256x256x256: 8 rows make only 256 CTAs and reach 0.55)
constexpr int MESH_ROWS_WIDE = 8, MESH_ROWS_NARROW = 2;

// Pass 1: a CTA marches MESH_KC layers of NR cube rows of one 256-column piece, one thread a
// column.  Each layer's NR + 1 cell rows are loaded and classified once (the inside bit of
// column i + 1 from the next lane's ballot), shared by the two cube rows each touches; a cube's count
// is a lookup by its 8-bit inside mask; the counts of each (layer, row, piece) segment are summed
// over the piece's warps.
template <typename R, int NR>
__global__ void __launch_bounds__(MESH_W) mesh_count_kernel(const Ph<R> *__restrict__ phi, const DevState *__restrict__ st,
                                                           int nx, int ny, int nz, int phase, R iso,
                                                           unsigned *__restrict__ seg_counts)
{
    constexpr int NL = NR + 1;  // cell rows the NR cube rows touch
    __shared__ unsigned wsum[MESH_KC][NR][MESH_W / 32];
    __shared__ unsigned char table[256];  // triangles of a cube by its inside mask
    table[threadIdx.x] = (unsigned char)mask_count((int)threadIdx.x);
    const int nb = (nx + MESH_W - 1) / MESH_W;
    const int b = blockIdx.x % nb, jg = blockIdx.x / nb, j0 = jg * NR;
    const int k0 = blockIdx.y * MESH_KC, k1 = min(nz - 1, k0 + MESH_KC);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = b * MESH_W + threadIdx.x;
    const bool act = i < nx;
    const int ic = act ? i : nx - 1;
    const int i1 = ic + 1 == nx ? 0 : ic + 1;
    const bool from_lane = lane < 31 && ic + 1 < nx;  // the next lane holds column i + 1
    const size_t plane = (size_t)nx * ny;
    const int zbase = st->zbase;
    // cell row r of the group: global row j0 + r, periodic
    int row[NL];
#pragma unroll
    for (int r = 0; r < NL; r++) row[r] = (j0 + r) % ny;
    auto ld = [&](int k, int jj, int ii) { return phi[plane_off(k, nz, zbase, plane) + (size_t)jj * nx + ii].v[phase]; };
    // the inside bits of a layer: bit r of lo / hi: cell (i, row r) / (i + 1, row r)
    struct Bits {
        unsigned a, b;
    };
    auto layer = [&](const R (&v)[NL], const R (&v1)[NL]) {
        Bits o{0u, 0u};
#pragma unroll
        for (int r = 0; r < NL; r++) {
            const bool in = v[r] >= iso;
            const unsigned m = __ballot_sync(0xffffffffu, in);
            const bool in1 = from_lane ? ((m >> (lane + 1)) & 1u) != 0 : v1[r] >= iso;
            o.a |= (unsigned)in << r;
            o.b |= (unsigned)in1 << r;
        }
        return o;
    };
    auto load = [&](int k, R (&v)[NL], R (&v1)[NL]) {
#pragma unroll
        for (int r = 0; r < NL; r++) {
            v[r] = ld(k, row[r], ic);
            v1[r] = v[r];
            if (!from_lane) v1[r] = ld(k, row[r], i1);
        }
    };
    R cv[NL], cv1[NL], qv[NL], qv1[NL];
    load(k0, cv, cv1);
    if (k0 + 1 <= k1) load(k0 + 1, qv, qv1);  // layer k + 1 in flight while layer k is classified
    Bits lo = layer(cv, cv1);
    __syncthreads();  // the table
    for (int k = k0; k < k1; k++) {
        const Bits hi = layer(qv, qv1);
        if (k + 2 <= k1) load(k + 2, qv, qv1);
#pragma unroll
        for (int r = 0; r < NR; r++) {
            // corners: 0 (i, j), 1 (i+1, j), 2 (i, j+1), 3 (i+1, j+1), then the same + 4 for layer k + 1
            const unsigned m = ((lo.a >> r) & 1u) | (((lo.b >> r) & 1u) << 1) | (((lo.a >> (r + 1)) & 1u) << 2) |
                               (((lo.b >> (r + 1)) & 1u) << 3) | (((hi.a >> r) & 1u) << 4) |
                               (((hi.b >> r) & 1u) << 5) | (((hi.a >> (r + 1)) & 1u) << 6) |
                               (((hi.b >> (r + 1)) & 1u) << 7);
            unsigned n = act && j0 + r < ny ? (unsigned)table[m] : 0u;
            n = __reduce_add_sync(0xffffffffu, n);
            if (lane == 0) wsum[k - k0][r][w] = n;
        }
        lo = hi;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < (k1 - k0) * NR; q += MESH_W) {
        const int kk = q / NR, r = q % NR;
        if (j0 + r >= ny) continue;
        unsigned sum = 0;
#pragma unroll
        for (int u = 0; u < MESH_W / 32; u++) sum += wsum[kk][r][u];
        seg_counts[((size_t)(k0 + kk) * ny + j0 + r) * nb + b] = sum;
    }
}

// exclusive block-wide sums of two per-thread values (1024 threads); returns the block totals
__device__ __forceinline__ void block_scan2(unsigned long long &x, unsigned &y, unsigned long long &tx, unsigned &ty,
                                            unsigned long long *sx, unsigned *sy)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long ix = x;
    unsigned iy = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long px = __shfl_up_sync(0xffffffffu, ix, o);
        const unsigned py = __shfl_up_sync(0xffffffffu, iy, o);
        if (lane >= o) {
            ix += px;
            iy += py;
        }
    }
    if (lane == 31) {
        sx[w] = ix;
        sy[w] = iy;
    }
    __syncthreads();
    if (w == 0) {
        unsigned long long vx = sx[lane];
        unsigned vy = sy[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long px = __shfl_up_sync(0xffffffffu, vx, o);
            const unsigned py = __shfl_up_sync(0xffffffffu, vy, o);
            if (lane >= o) {
                vx += px;
                vy += py;
            }
        }
        sx[lane] = vx;  // inclusive over warps
        sy[lane] = vy;
    }
    __syncthreads();
    const unsigned long long bx = w ? sx[w - 1] : 0ull;
    const unsigned by = w ? sy[w - 1] : 0u;
    x = bx + ix - x;
    y = by + iy - y;
    tx = sx[31];
    ty = sy[31];
    __syncthreads();
}

// pass 2: one CTA of 1024 threads over the segment counts (padded with zeros to a multiple of 16):
// the offsets and ids of the non-empty segments, and the totals (triangles, non-empty segments)
static __global__ void __launch_bounds__(1024) mesh_scan_kernel(const unsigned *__restrict__ seg_counts, size_t nseg_pad,
                                                         unsigned *__restrict__ ne_seg,
                                                         unsigned long long *__restrict__ ne_off,
                                                         unsigned long long *__restrict__ totals)
{
    __shared__ unsigned long long sx[32];
    __shared__ unsigned sy[32];
    unsigned long long carry = 0;
    unsigned ncarry = 0;
    for (size_t base = 0; base < nseg_pad; base += 1024 * 16) {
        const size_t first = base + (size_t)threadIdx.x * 16;
        unsigned v[16];
        if (first < nseg_pad) {
            const uint4 *p4 = reinterpret_cast<const uint4 *>(seg_counts + first);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint4 u = p4[q];
                v[4 * q] = u.x;
                v[4 * q + 1] = u.y;
                v[4 * q + 2] = u.z;
                v[4 * q + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] = 0;
        }
        unsigned long long sum = 0;
        unsigned ne = 0;
#pragma unroll
        for (int q = 0; q < 16; q++) {
            sum += v[q];
            ne += v[q] ? 1u : 0u;
        }
        unsigned long long tsum;
        unsigned tne;
        block_scan2(sum, ne, tsum, tne, sx, sy);
        unsigned long long off = carry + sum;
        unsigned pos = ncarry + ne;
#pragma unroll
        for (int q = 0; q < 16; q++) {
            if (v[q]) {
                ne_seg[pos] = (unsigned)(first + q);
                ne_off[pos] = off;
                pos++;
                off += v[q];
            }
        }
        carry += tsum;
        ncarry += tne;
    }
    if (threadIdx.x == 0) {
        totals[0] = carry;
        totals[1] = ncarry;
    }
}

// pass 3: the triangles of each listed segment, from its offset, in cube order.  The crossed cubes
// of the segment are gathered into shared memory, then the CTA's threads take one (cube,
// tetrahedron) pair each, so that the lanes stay busy however sparse the crossed cubes are.
template <typename R>
__global__ void __launch_bounds__(MESH_W) mesh_emit_kernel(const Ph<R> *__restrict__ phi, const DevState *__restrict__ st,
                                                          int nx, int ny, int nz, int phase, R iso,
                                                          const unsigned *__restrict__ ne_seg,
                                                          const unsigned long long *__restrict__ ne_off,
                                                          unsigned long long total, float *__restrict__ out)
{
    __shared__ unsigned ws[MESH_W / 32], wc[MESH_W / 32];
    __shared__ R sf[MESH_W][8];
    __shared__ unsigned s_first[MESH_W];  // first triangle of the crossed cube, relative to the segment
    __shared__ int s_i[MESH_W];
    const int nb = (nx + MESH_W - 1) / MESH_W;
    const size_t seg = ne_seg[blockIdx.x];
    const int b = (int)(seg % nb), j = (int)((seg / nb) % ny), k = (int)(seg / ((size_t)nb * ny));
    const int i = b * MESH_W + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    R f[8];
    unsigned n = 0;
    if (i < nx) {
        corner_values(phi, nx, ny, nz, st->zbase, phase, i, j, k, f);
        n = (unsigned)cube_count(f, iso);
    }
    // exclusive prefixes over the segment of the triangles and of the crossed cubes
    unsigned x = n, c = n ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o), z = __shfl_up_sync(0xffffffffu, c, o);
        if (lane >= o) {
            x += y;
            c += z;
        }
    }
    if (lane == 31) {
        ws[w] = x;
        wc[w] = c;
    }
    __syncthreads();
    unsigned before = 0, cbefore = 0, ncross = 0;
    for (int q = 0; q < MESH_W / 32; q++) {
        if (q < w) {
            before += ws[q];
            cbefore += wc[q];
        }
        ncross += wc[q];
    }
    if (n) {
        const unsigned slot = cbefore + c - 1;
#pragma unroll
        for (int m = 0; m < 8; m++) sf[slot][m] = f[m];
        s_first[slot] = before + x - n;
        s_i[slot] = i;
    }
    __syncthreads();
    const unsigned long long seg_first = ne_off[blockIdx.x];
    const R by = (R)j + (R)0.5, bz = (R)k + (R)0.5 + (R)st->off;
    for (unsigned item = threadIdx.x; item < ncross * 6; item += MESH_W) {
        const unsigned slot = item / 6;
        const int q = (int)(item - slot * 6);
        R g[8];
#pragma unroll
        for (int m = 0; m < 8; m++) g[m] = sf[slot][m];
        unsigned first = s_first[slot];
        for (int p = 0; p < q; p++) first += (unsigned)tet_count(g, p, iso);
        const unsigned long long at = seg_first + first;
        if (at + (unsigned long long)tet_count(g, q, iso) <= total)  // the counts of pass 1 and here agree; the bound guards the buffer
            tet_emit(g, q, iso, (R)s_i[slot] + (R)0.5, by, bz, out + 9ull * at);
    }
}

}  // namespace pf
