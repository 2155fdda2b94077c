// Several DD problems stepped together.
//
// One batched iteration of solves s = 1..S on one data set:
//   * P_C: gather, right-hand sides and recovery per solve, and ONE
//     cooperative launch that runs the mixed-precision CG of every solve:
//     each solve owns a contiguous range of thread blocks, reduces its dot
//     products over that range only (fixed order), and all solves share the
//     grid barriers; a solve that has converged idles until the others have;
//   * P_D: ONE search over the concatenated states of all solves (the
//     per-material-point search is independent of the solve it belongs to),
//     with per-query f_d for the approximate search, whose ramp depends on
//     each solve's own iteration count;
//   * statistics and the stop rule per solve.
// Solves can have meshes of different sizes; they share the search mode and
// the CG mode.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dd_internal.cuh"
#include "fem.cuh"
#include "fem_dev.cuh"
#include "solver.cuh"

namespace {

// The product K v runs on node tiles of tx x ty x tz free nodes (k >= 1: the
// clamped face carries no unknowns, and every vector is zero there): the
// block stages the tile and a one-node halo of v in shared memory, and every
// thread applies the 27-point stencil of its node (fem_stencil_table) from
// there, with the 3x3 blocks of its boundary class.
//
// The inner FP32 iterations are preconditioned by one multigrid V-cycle
// (trilinear spaces with the element size doubled per level, so that the
// operator of level l is 2^l K of level 0; restriction is the transpose of
// trilinear prolongation) with one damped block-Jacobi sweep before and after
// the coarse correction; the coarsest level is solved exactly with a dense
// inverse shared out over the blocks of each solve.  A solve whose mesh cannot
// coarsen uses block-Jacobi alone.
constexpr int kBThreads = 256;
constexpr int kTileMax = 16;                 // tile edge bound (nodes)
constexpr int kHaloMax = 1024;               // (tx + 2)(ty + 2)(tz + 2) bound
constexpr int kSt32 = 27 * 27 * 12;          // FP32 stencil table (floats)
constexpr size_t kSmemSt = (size_t)kSt32 * 4;
constexpr size_t kSmemHalo = (size_t)kHaloMax * 6 * 8;
constexpr size_t kSmemLev = (size_t)(kMgDirectDofs / 3 + 1) * 6 * 4;
constexpr size_t kSmemDi = 27 * 6 * 4 + 16;
constexpr size_t kDynSmem = kSmemSt + kSmemHalo + kSmemLev + kSmemDi;

struct Level {
    int nx, ny, nz;                          // elements
    int top;                                 // 1: the top layer of nodes is fixed (free layers 1 .. nz - top)
    int tx, ty, tz, ntx, nty, ntiles;        // tiles (levels run by the whole grid)
    float *r, *z, *t;                        // vectors [nodes x 6] (grid levels)
    float h;                                 // 2^level
};

struct SegCG {
    const double *St64, *b;
    const float *St32;
    double *x;
    float *r, *z, *p0, *p1, *q, *d;
    float *zg;                               // solution of the coarsest level (all its nodes)
    const float *inv;                        // dense inverse of the coarsest level's K
    int ndof;                                // its free DOFs
    int blk0, nblk;
    int nlev, glev;
    float omega;
    Level lv[kMgMaxLev];
};

struct BCGArgs {
    const SegCG *seg;
    const int *blk_seg;        // [grid] solve of every block
    int S;
    int G;                     // largest number of grid levels over the solves
    double *part;              // [2 x grid x 8]
    int *flags;                // [S]: outer activity (written by segment leaders)
    unsigned *bar, *err;
    double rtol2, in_rtol2;
    int max_outer, max_inner;
    int *it_out;               // [S] inner iterations of every solve
};

// Sum over the partials of blocks [b0, b0 + nb) in a fixed order.
template <int NV>
__device__ void range_total(const double *part, int b0, int nb, double (&tot)[NV], double *sh) {
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] += __ldcg(part + (size_t)(b0 + t) * 8 + c);
    block_sum<NV>(v, sh);
    __shared__ double s_tot[8];
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) s_tot[c] = v[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NV; ++c) tot[c] = s_tot[c];
    __syncthreads();
}

// Slots [0, NV) summed over the blocks [b0, b0 + nb) of this solve, slot 7
// (activity) summed over all G blocks and slot 6 (multigrid depth) maxed over
// them, in one fixed-order pass.  Returns the activity; *gmax the depth.
template <int NV>
__device__ double seg_totals(const double *part, int G, int b0, int nb, double (&tot)[NV], double *sh, int *gmax) {
    double v[NV + 1];
    int gm = 0;
#pragma unroll
    for (int c = 0; c <= NV; ++c) v[c] = 0.0;
    for (int t = threadIdx.x; t < G; t += blockDim.x) {
        if (t >= b0 && t < b0 + nb)
#pragma unroll
            for (int c = 0; c < NV; ++c) v[c] += __ldcg(part + (size_t)t * 8 + c);
        v[NV] += __ldcg(part + (size_t)t * 8 + 7);
        gm = max(gm, (int)__ldcg(part + (size_t)t * 8 + 6));
    }
    for (int o = 16; o > 0; o >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    __shared__ int s_gm[32];
    if ((threadIdx.x & 31) == 0) s_gm[threadIdx.x >> 5] = gm;
    block_sum<NV + 1>(v, sh);
    __shared__ double s_tot[8];
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c <= NV; ++c) s_tot[c] = v[c];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s_gm[0] = max(s_gm[0], s_gm[w]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NV; ++c) tot[c] = s_tot[c];
    const double all = s_tot[NV];
    *gmax = s_gm[0];
    __syncthreads();
    return all;
}

// Sum and maximum of the per-solve flags (written by the solve leaders).
__device__ void flag_stats(const int *flags, int S, double *sh, int *sum, int *mx) {
    int c = 0, m = 0;
    for (int t = threadIdx.x; t < S; t += blockDim.x) {
        const int f = __ldcg(flags + t);
        c += f > 0;
        m = max(m, f);
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    __shared__ int s_c[32], s_m[32];
    if ((threadIdx.x & 31) == 0) {
        s_c[threadIdx.x >> 5] = c;
        s_m[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            s_c[0] += s_c[w];
            s_m[0] = max(s_m[0], s_m[w]);
        }
    __syncthreads();
    *sum = s_c[0];
    *mx = s_m[0];
    __syncthreads();
    (void)sh;
}

__device__ __forceinline__ int lnode(const Level L, int X, int Y, int Z) { return X + (L.nx + 1) * (Y + (L.ny + 1) * Z); }

__device__ __forceinline__ int lclass(const Level L, int X, int Y, int Z) {
    const int cx = X == 0 ? 0 : (X == L.nx ? 2 : 1);
    const int cy = Y == 0 ? 0 : (Y == L.ny ? 2 : 1);
    const int cz = Z == L.nz ? 2 : 1;
    return cx + 3 * cy + 9 * cz;
}

// This thread's place in a tile of level L, and the decomposition of its
// halo slots h = threadIdx.x + k * kBThreads (packed x | y << 8 | z << 16).
struct Lane {
    int lx, ly, lz, hx, hxy, hc, nh;
    bool ok;
    int hs[4];
};

__device__ __forceinline__ Lane lane_of(const Level L) {
    Lane n;
    const int t = threadIdx.x;
    n.ok = t < L.tx * L.ty * L.tz;
    n.lx = t % L.tx;
    n.ly = (t / L.tx) % L.ty;
    n.lz = t / (L.tx * L.ty);
    n.hx = L.tx + 2;
    n.hxy = n.hx * (L.ty + 2);
    n.hc = (n.lx + 1) + n.hx * (n.ly + 1) + n.hxy * (n.lz + 1);
    n.nh = n.hxy * (L.tz + 2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int h = t + k * kBThreads;
        n.hs[k] = (h % n.hx) | (((h / n.hx) % (L.ty + 2)) << 8) | ((h / n.hxy) << 16);
    }
    return n;
}

// This thread's node in tile `tile` of level L.
struct TileNode {
    int X0, Y0, Z0;   // tile origin
    int a;            // node id
    int cls;          // stencil class
    bool ok;
};

__device__ __forceinline__ TileNode tile_node(const Level L, const Lane &ln, int tile) {
    TileNode n;
    n.X0 = (tile % L.ntx) * L.tx;
    n.Y0 = ((tile / L.ntx) % L.nty) * L.ty;
    n.Z0 = 1 + (tile / (L.ntx * L.nty)) * L.tz;
    const int X = n.X0 + ln.lx, Y = n.Y0 + ln.ly, Z = n.Z0 + ln.lz;
    n.ok = ln.ok && X <= L.nx && Y <= L.ny && Z <= L.nz - L.top;
    n.a = n.ok ? lnode(L, X, Y, Z) : 0;
    n.cls = lclass(L, X, Y, Z);
    return n;
}

// sv[h] = vz + beta .* vp (vp may be null) at every node h of the tile's
// halo; nodes outside the box or on the clamped face hold 0.  All loads of a
// thread are issued before its stores.
__device__ __forceinline__ void stage_f(const Level L, const Lane &ln, const TileNode &n, const float *vz,
                                        const float *vp, const float beta[2], float *sv) {
    float2 v[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int h = threadIdx.x + k * kBThreads;
        const int X = n.X0 - 1 + (ln.hs[k] & 255), Y = n.Y0 - 1 + ((ln.hs[k] >> 8) & 255),
                  Z = n.Z0 - 1 + (ln.hs[k] >> 16);
        v[k][0] = v[k][1] = v[k][2] = make_float2(0.f, 0.f);
        if (h < ln.nh && X >= 0 && Y >= 0 && Z >= 1 && X <= L.nx && Y <= L.ny && Z <= L.nz - L.top) {
            const int a = lnode(L, X, Y, Z);
            const float2 *pz = reinterpret_cast<const float2 *>(vz + (size_t)a * 6);
            v[k][0] = __ldcg(pz);
            v[k][1] = __ldcg(pz + 1);
            v[k][2] = __ldcg(pz + 2);
            if (vp) {
                const float2 *pp = reinterpret_cast<const float2 *>(vp + (size_t)a * 6);
                const float2 w0 = __ldcg(pp), w1 = __ldcg(pp + 1), w2 = __ldcg(pp + 2);
                v[k][0].x = fmaf(beta[0], w0.x, v[k][0].x);
                v[k][0].y = fmaf(beta[0], w0.y, v[k][0].y);
                v[k][1].x = fmaf(beta[0], w1.x, v[k][1].x);
                v[k][1].y = fmaf(beta[1], w1.y, v[k][1].y);
                v[k][2].x = fmaf(beta[1], w2.x, v[k][2].x);
                v[k][2].y = fmaf(beta[1], w2.y, v[k][2].y);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int h = threadIdx.x + k * kBThreads;
        if (h < ln.nh) {
            float2 *o = reinterpret_cast<float2 *>(sv + h * 6);
            o[0] = v[k][0];
            o[1] = v[k][1];
            o[2] = v[k][2];
        }
    }
}

__device__ __forceinline__ void stage_d(const Level L, const Lane &ln, const TileNode &n, const double *vz,
                                        double *sv) {
    for (int h = threadIdx.x; h < ln.nh; h += blockDim.x) {
        const int X = n.X0 - 1 + h % ln.hx, Y = n.Y0 - 1 + (h / ln.hx) % (L.ty + 2), Z = n.Z0 - 1 + h / ln.hxy;
        double2 v0 = make_double2(0.0, 0.0), v1 = v0, v2 = v0;
        if (X >= 0 && Y >= 0 && Z >= 1 && X <= L.nx && Y <= L.ny && Z <= L.nz) {
            const double2 *pz = reinterpret_cast<const double2 *>(vz + (size_t)lnode(L, X, Y, Z) * 6);
            v0 = __ldcg(pz);
            v1 = __ldcg(pz + 1);
            v2 = __ldcg(pz + 2);
        }
        double2 *o = reinterpret_cast<double2 *>(sv + h * 6);
        o[0] = v0;
        o[1] = v1;
        o[2] = v2;
    }
}

// y += (3x3 block kb) applied to both systems of the node values xv.
__device__ __forceinline__ void block_apply(const float *Sc, int d, const float *xv, float y[6]) {
    const float2 *x2 = reinterpret_cast<const float2 *>(xv);
    const float2 x01 = x2[0], x23 = x2[1], x45 = x2[2];
    const float4 *kb = reinterpret_cast<const float4 *>(Sc + d * 12);
    const float4 k0 = kb[0], k1 = kb[1], k2 = kb[2];
    // rows (k0.x k0.y k0.z), (k0.w k1.x k1.y), (k1.z k1.w k2.x)
    y[0] = fmaf(k0.x, x01.x, fmaf(k0.y, x01.y, fmaf(k0.z, x23.x, y[0])));
    y[1] = fmaf(k0.w, x01.x, fmaf(k1.x, x01.y, fmaf(k1.y, x23.x, y[1])));
    y[2] = fmaf(k1.z, x01.x, fmaf(k1.w, x01.y, fmaf(k2.x, x23.x, y[2])));
    y[3] = fmaf(k0.x, x23.y, fmaf(k0.y, x45.x, fmaf(k0.z, x45.y, y[3])));
    y[4] = fmaf(k0.w, x23.y, fmaf(k1.x, x45.x, fmaf(k1.y, x45.y, y[4])));
    y[5] = fmaf(k1.z, x23.y, fmaf(k1.w, x45.x, fmaf(k2.x, x45.y, y[5])));
}

// (K v) of the node at halo index hc, FP32 (level-0 table).
__device__ __forceinline__ void stencil_f(const float *sS, const float *sv, int hc, int hx, int hxy, int cls,
                                          float y[6]) {
    const float *Sc = sS + cls * (27 * 12);
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] = 0.f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx)
                block_apply(Sc, (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1), sv + (hc + dx + dy * hx + dz * hxy) * 6, y);
}

// The same in FP64 with the table read through the read-only cache.
__device__ __forceinline__ void stencil_d(const double *St, const double *sv, int hc, int hx, int hxy, int cls,
                                          double y[6]) {
    const double *Sc = St + cls * (27 * 9);
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] = 0.0;
#pragma unroll 1
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int d = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                const double *xv = sv + (hc + dx + dy * hx + dz * hxy) * 6;
                double k9[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) k9[k] = __ldg(Sc + d * 9 + k);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    y[r] = fma(k9[3 * r], xv[0], fma(k9[3 * r + 1], xv[1], fma(k9[3 * r + 2], xv[2], y[r])));
                    y[3 + r] = fma(k9[3 * r], xv[3], fma(k9[3 * r + 1], xv[4], fma(k9[3 * r + 2], xv[5], y[3 + r])));
                }
            }
}

// The part of (K v) of the node at halo index hc from its 9 neighbours in
// the layer above (dz = +1), FP64.
__device__ __forceinline__ void stencil_d_up(const double *St, const double *sv, int hc, int hx, int hxy, int cls,
                                             double y[6]) {
    const double *Sc = St + cls * (27 * 9);
#pragma unroll
    for (int k = 0; k < 6; ++k) y[k] = 0.0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int d = (dx + 1) + 3 * (dy + 1) + 18;
            const double *xv = sv + (hc + dx + dy * hx + hxy) * 6;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double k0 = __ldg(Sc + d * 9 + 3 * r), k1 = __ldg(Sc + d * 9 + 3 * r + 1),
                             k2 = __ldg(Sc + d * 9 + 3 * r + 2);
                y[r] = fma(k0, xv[0], fma(k1, xv[1], fma(k2, xv[2], y[r])));
                y[3 + r] = fma(k0, xv[3], fma(k1, xv[4], fma(k2, xv[5], y[3 + r])));
            }
        }
}

// y = s * D^-1 x for both systems, D^-1 of class cls packed (m00 m11 m22 m12 m02 m01).
__device__ __forceinline__ void dinv_apply(const float *sDi, int cls, float s, const float x[6], float y[6]) {
    const float *m = sDi + cls * 6;
    const float m00 = m[0] * s, m11 = m[1] * s, m22 = m[2] * s, m12 = m[3] * s, m02 = m[4] * s, m01 = m[5] * s;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float r0 = x[3 * q], r1 = x[3 * q + 1], r2 = x[3 * q + 2];
        y[3 * q + 0] = fmaf(m00, r0, fmaf(m01, r1, m02 * r2));
        y[3 * q + 1] = fmaf(m01, r0, fmaf(m11, r1, m12 * r2));
        y[3 * q + 2] = fmaf(m02, r0, fmaf(m12, r1, m22 * r2));
    }
}

__device__ __forceinline__ void ld6(const float *p, float v[6]) {
    const float2 *q = reinterpret_cast<const float2 *>(p);
    const float2 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

__device__ __forceinline__ void st6(float *p, const float v[6]) {
    float2 *q = reinterpret_cast<float2 *>(p);
    q[0] = make_float2(v[0], v[1]);
    q[1] = make_float2(v[2], v[3]);
    q[2] = make_float2(v[4], v[5]);
}

__device__ __forceinline__ float dot3(const float *a, const float *b) {
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

// r_C = sum over the fine nodes around 2C of the trilinear weights times t
// (restriction = transpose of prolongation); fine nodes outside the box or
// on the clamped face contribute 0.  get(a, v) reads the 6 values of fine
// node a; the loops are unrolled so that all 27 gathers are issued together.
template <typename Get>
__device__ __forceinline__ void restrict_node(const Level F, int X, int Y, int Z, Get get, float r[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) r[k] = 0.f;
#pragma unroll
    for (int pz = 0; pz < 3; ++pz) {   // one plane of 9 fine nodes per round of gathers
        const int z = 2 * Z + pz - 1;
        float v[9][6];
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const int x = 2 * X + d % 3 - 1, y = 2 * Y + d / 3 - 1;
            if (x >= 0 && y >= 0 && z >= 1 && x <= F.nx && y <= F.ny && z <= F.nz - F.top) {
                get(lnode(F, x, y, z), v[d]);
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) v[d][k] = 0.f;
            }
        }
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const float w = (d % 3 == 1 ? 1.f : 0.5f) * (d / 3 == 1 ? 1.f : 0.5f) * (pz == 1 ? 1.f : 0.5f);
#pragma unroll
            for (int k = 0; k < 6; ++k) r[k] = fmaf(w, v[d][k], r[k]);
        }
    }
}

// e_f = sum over the (up to 8) coarse nodes of fine node (X, Y, Z) of the
// trilinear weights times the coarse values; coarse nodes on the clamped face
// hold 0.  get(A, v) reads the 6 values of coarse node A.
template <typename Get>
__device__ __forceinline__ void prolong_node(const Level Cl, int X, int Y, int Z, Get get, float e[6]) {
    const int I[2] = {X >> 1, (X + 1) >> 1}, J[2] = {Y >> 1, (Y + 1) >> 1}, K[2] = {Z >> 1, (Z + 1) >> 1};
    const float wx = (X & 1) ? 0.5f : 1.f, wy = (Y & 1) ? 0.5f : 1.f, wz = (Z & 1) ? 0.5f : 1.f;
    float v[8][6];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        // odd coordinates take both neighbours, even ones the coincident node once
        const bool use = (c & 1 ? (X & 1) : 1) && (c & 2 ? (Y & 1) : 1) && (c & 4 ? (Z & 1) : 1) &&
                         K[(c >> 2) & 1] >= 1 && K[(c >> 2) & 1] <= Cl.nz - Cl.top;
        if (use) {
            get(lnode(Cl, I[c & 1], J[(c >> 1) & 1], K[(c >> 2) & 1]), v[c]);
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) v[c][k] = 0.f;
        }
    }
    const float w = wx * wy * wz;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc += v[c][k];
        e[k] = w * acc;
    }
}

// ---- the coarsest level, solved exactly by all blocks of the solve ----

// Every block restricts the residual t of the last grid level to the free
// nodes of the coarsest level (its own shared-memory copy); the rows of the
// dense inverse are shared out over the solve's warps (one row per warp,
// lanes over the columns), and each row's two outputs (both systems) go to
// S.zg.  Block 0 also zeroes the clamped nodes.
__device__ void coarse_direct(const SegCG &S, int lb, int nblk, float *sr) {
    const int g = S.glev;
    const Level F = S.lv[g - 1], Cl = S.lv[g];
    const int plane = (Cl.nx + 1) * (Cl.ny + 1), nfree = plane * (Cl.nz - Cl.top), n = S.ndof;
    const float *tf = F.t;
    for (int f = threadIdx.x; f < nfree; f += blockDim.x) {
        const int a = plane + f;
        const int X = a % (Cl.nx + 1), Y = (a / (Cl.nx + 1)) % (Cl.ny + 1), Z = a / plane;
        float v[6];
        restrict_node(F, X, Y, Z, [&](int b, float *o) { ld6(tf + (size_t)b * 6, o); }, v);
#pragma unroll
        for (int k = 0; k < 6; ++k) sr[f * 6 + k] = v[k];
    }
    __syncthreads();
    const float *inv = S.inv;
    float *zg = S.zg;
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    for (int i = lb * warps + (threadIdx.x >> 5); i < n; i += nblk * warps) {
        float a0 = 0.f, a1 = 0.f;
        for (int j = lane; j < n; j += 32) {   // K^-1 is symmetric: row i
            const float A = __ldg(inv + (size_t)i * n + j);
            const float *rj = sr + (j / 3) * 6 + j % 3;
            a0 = fmaf(A, rj[0], a0);
            a1 = fmaf(A, rj[3], a1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (lane == 0) {
            const int fi = i / 3, ci = i % 3;
            zg[(size_t)(plane + fi) * 6 + ci] = a0;
            zg[(size_t)(plane + fi) * 6 + 3 + ci] = a1;
        }
    }
    if (lb == 0) {   // fixed nodes: the bottom plane, and the top plane when it is fixed
        for (int k = threadIdx.x; k < plane * 6; k += blockDim.x) zg[k] = 0.f;
        if (Cl.top)
            for (int k = threadIdx.x; k < plane * 6; k += blockDim.x) zg[(size_t)plane * Cl.nz * 6 + k] = 0.f;
    }
}

// ---- grid-level operations (all blocks of the solve, node tiles) ----

// t = r - h K z at grid level l.
__device__ void grid_residual(const Level L, int lb, int nblk, const float *sS, float *sv) {
    const Lane ln = lane_of(L);
    const float zb[2] = {0.f, 0.f};
    for (int tile = lb; tile < L.ntiles; tile += nblk) {
        const TileNode n = tile_node(L, ln, tile);
        __syncthreads();
        stage_f(L, ln, n, L.z, nullptr, zb, sv);
        __syncthreads();
        if (n.ok) {
            float kz[6], rv[6];
            stencil_f(sS, sv, ln.hc, ln.hx, ln.hxy, n.cls, kz);
            ld6(L.r + (size_t)n.a * 6, rv);
#pragma unroll
            for (int k = 0; k < 6; ++k) kz[k] = fmaf(-L.h, kz[k], rv[k]);
            st6(L.t + (size_t)n.a * 6, kz);
        }
    }
}

// z = t + omega / h D^-1 (r - h K t) at grid level l (t holds z + P e);
// level 0 also accumulates (r.z, r.r) of both systems.
__device__ void grid_post_smooth(const Level L, int lb, int nblk, const float *sS, const float *sDi, float om,
                                 float *sv, double (&dots)[4]) {
    const Lane ln = lane_of(L);
    const float zb[2] = {0.f, 0.f};
    for (int tile = lb; tile < L.ntiles; tile += nblk) {
        const TileNode n = tile_node(L, ln, tile);
        __syncthreads();
        stage_f(L, ln, n, L.t, nullptr, zb, sv);
        __syncthreads();
        if (n.ok) {
            float kz[6], rv[6], zv[6], dz[6];
            stencil_f(sS, sv, ln.hc, ln.hx, ln.hxy, n.cls, kz);
            ld6(L.r + (size_t)n.a * 6, rv);
#pragma unroll
            for (int k = 0; k < 6; ++k) kz[k] = fmaf(-L.h, kz[k], rv[k]);
            dinv_apply(sDi, n.cls, om / L.h, kz, dz);
            const float *own = sv + ln.hc * 6;
#pragma unroll
            for (int k = 0; k < 6; ++k) zv[k] = own[k] + dz[k];
            st6(L.z + (size_t)n.a * 6, zv);
            dots[0] += (double)dot3(rv, zv);
            dots[1] += (double)dot3(rv + 3, zv + 3);
            dots[2] += (double)dot3(rv, rv);
            dots[3] += (double)dot3(rv + 3, rv + 3);
        }
    }
}

// Coarse level C = l + 1 run by the grid: r_C = P^T t_l, z_C = omega / h D^-1 r_C.
__device__ void grid_restrict(const Level F, const Level C, int lb, int nblk, const float *sDi, float om) {
    const Lane ln = lane_of(C);
    for (int tile = lb; tile < C.ntiles; tile += nblk) {
        const TileNode n = tile_node(C, ln, tile);
        if (!n.ok) continue;
        const int X = n.X0 + ln.lx, Y = n.Y0 + ln.ly, Z = n.Z0 + ln.lz;
        float rv[6], zv[6];
        restrict_node(F, X, Y, Z, [&](int b, float *o) { ld6(F.t + (size_t)b * 6, o); }, rv);
        dinv_apply(sDi, n.cls, om / C.h, rv, zv);
        st6(C.r + (size_t)n.a * 6, rv);
        st6(C.z + (size_t)n.a * 6, zv);
    }
}

// t_l = z_l + P z_C at grid level l (zc: the coarse correction, all nodes of C).
__device__ void grid_prolong(const Level L, const Level C, const float *zc, int lb, int nblk) {
    const Lane ln = lane_of(L);
    for (int tile = lb; tile < L.ntiles; tile += nblk) {
        const TileNode n = tile_node(L, ln, tile);
        if (!n.ok) continue;
        const int X = n.X0 + ln.lx, Y = n.Y0 + ln.ly, Z = n.Z0 + ln.lz;
        float e[6], zv[6];
        if (zc) {
            prolong_node(C, X, Y, Z, [&](int b, float *o) { ld6(zc + (size_t)b * 6, o); }, e);
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) e[k] = 0.f;
        }
        ld6(L.z + (size_t)n.a * 6, zv);
#pragma unroll
        for (int k = 0; k < 6; ++k) zv[k] += e[k];
        st6(L.t + (size_t)n.a * 6, zv);
    }
}

// The rest of one V-cycle after the level-0 pre-smoothing z_0 = omega D^-1 r
// (done by the caller and followed by a grid barrier): residual and
// restriction down the grid levels, the exact coarse solve, prolongation and
// post-smoothing back up.  Every block passes the same 4 G - 1 barriers;
// blocks of a solve that is inactive or has fewer grid levels only wait.
// The final level-0 post-smoothing writes S.z and this block's (r.z, r.r).
__device__ bool vcycle_rest(const SegCG &S, int lb, bool act, int G, GridBar &gb, unsigned *err, const float *sS,
                            const float *sDi, float *sv, float *sLev, double (&dots)[4]) {
    const float om = S.omega;
    const int glev = S.glev, nlev = S.nlev, nblk = S.nblk;
    const float *const zg = S.zg;
    for (int l = 0; l < G; ++l) {
        if (act && l < glev) grid_residual(S.lv[l], lb, nblk, sS, sv);
        if (!grid_sync(gb, err)) return false;
        if (act && l + 1 < glev) grid_restrict(S.lv[l], S.lv[l + 1], lb, nblk, sDi, om);
        if (act && l + 1 == glev && glev < nlev) coarse_direct(S, lb, nblk, sLev);
        if (!grid_sync(gb, err)) return false;
    }
    for (int l = G - 1; l >= 0; --l) {
        if (act && l < glev) {
            const float *zc = l + 1 < glev ? S.lv[l + 1].z : (l + 1 < nlev ? zg : nullptr);
            grid_prolong(S.lv[l], S.lv[l + 1 < nlev ? l + 1 : l], zc, lb, nblk);
        }
        if (!grid_sync(gb, err)) return false;
        if (act && l < glev) {
            double dd[4] = {0, 0, 0, 0};
            grid_post_smooth(S.lv[l], lb, nblk, sS, sDi, om, sv, l == 0 ? dots : dd);
        }
        if (l > 0 && !grid_sync(gb, err)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kBThreads, 1) k_cg_batch(BCGArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    float *sS = reinterpret_cast<float *>(dsm);                                  // [kSt32]
    double *sv64 = reinterpret_cast<double *>(dsm + kSmemSt);                     // [kHaloMax x 6]
    float *sv32 = reinterpret_cast<float *>(sv64);                               // the FP32 halo reuses it
    float *sLev = reinterpret_cast<float *>(dsm + kSmemSt + kSmemHalo);           // coarse residual
    float *sDi = reinterpret_cast<float *>(dsm + kSmemSt + kSmemHalo + kSmemLev); // [27 x 6]
    __shared__ double sh[8 * 32];
    const int sidx = A.blk_seg[blockIdx.x];
    const SegCG &S = A.seg[sidx];
    for (int t = threadIdx.x; t < kSt32 / 4; t += blockDim.x)
        reinterpret_cast<float4 *>(sS)[t] = __ldg(reinterpret_cast<const float4 *>(S.St32) + t);
    __syncthreads();
    if (threadIdx.x < 27) {   // inverse of the diagonal block of every class, packed symmetric
        const float *D = sS + (threadIdx.x * 27 + 13) * 12;
        const float d00 = D[0], d01 = D[1], d02 = D[2], d11 = D[4], d12 = D[5], d22 = D[8];
        const float c00 = d11 * d22 - d12 * d12, c01 = d02 * d12 - d01 * d22, c02 = d01 * d12 - d02 * d11;
        const float det = d00 * c00 + d01 * c01 + d02 * c02;
        const float id = 1.f / det;
        float *m = sDi + threadIdx.x * 6;
        m[0] = c00 * id;
        m[1] = (d00 * d22 - d02 * d02) * id;
        m[2] = (d00 * d11 - d01 * d01) * id;
        m[3] = (d01 * d02 - d00 * d12) * id;
        m[4] = c02 * id;
        m[5] = c01 * id;
    }
    __syncthreads();
    const unsigned G = gridDim.x;
    GridBar gbar{A.bar, G, 0u};
    const int lb = blockIdx.x - S.blk0;
    const bool leader = (lb == 0 && threadIdx.x == 0);
    const Level L0 = S.lv[0];
    const Lane ln0 = lane_of(L0);
    const float om = S.omega;
    const int nblk = S.nblk, blk0 = S.blk0;
    float *const Sr = S.r, *const Sz = S.z, *const Sd = S.d, *const Sq = S.q;
    double *const Sx = S.x;
    const double *const Sb = S.b, *const St64 = S.St64;
    const double ndof = 3.0 * (L0.nx + 1) * (double)(L0.ny + 1) * (double)(L0.nz - L0.top);
    double *partA = A.part, *partB = A.part + (size_t)G * 8;
    int *outer_flag = A.flags;
    // multigrid depth of this solve (0: one level, plain block-Jacobi)
    const int gdepth = S.nlev > 1 ? S.glev : 0;
    int inner_count = 0;
    for (int outer = 0;; ++outer) {
        // ---- FP64 residual r = b - K x and the norms ----
        double v[4] = {0, 0, 0, 0};   // r.r (2), b.b (2)
        for (int tile = lb; tile < L0.ntiles; tile += nblk) {
            const TileNode n = tile_node(L0, ln0, tile);
            __syncthreads();
            stage_d(L0, ln0, n, Sx, sv64);
            __syncthreads();
            if (n.ok) {
                const size_t a = n.a;
                double kx[6], lift[6] = {0, 0, 0, 0, 0, 0};
                stencil_d(St64, sv64, ln0.hc, ln0.hx, ln0.hxy, n.cls, kx);
                // below a fixed top: the coupling to the prescribed values, which
                // moves to the right-hand side of the free dofs (the reference norm)
                if (L0.top && n.Z0 + ln0.lz == L0.nz - 1) stencil_d_up(St64, sv64, ln0.hc, ln0.hx, ln0.hxy, n.cls, lift);
                float rf[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const double bc = Sb[a * 6 + k];
                    const double r64 = bc - kx[k];
                    rf[k] = (float)r64;
                    v[k / 3] += r64 * r64;
                    v[2 + k / 3] += (bc - lift[k]) * (bc - lift[k]);
                }
                st6(Sr + a * 6, rf);
                const float zero6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                st6(Sd + a * 6, zero6);
            }
        }
        block_sum<4>(v, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 4; ++k) partB[blockIdx.x * 8 + k] = v[k];
        if (!grid_sync(gbar, A.err)) return;
        double tot[4];
        range_total<4>(partB, blk0, nblk, tot, sh);
        double rr_true[2], bb[2], scale[2], unscale[2];
        bool conv[2];
        for (int s2 = 0; s2 < 2; ++s2) {
            rr_true[s2] = tot[s2];
            bb[s2] = tot[2 + s2];
            conv[s2] = !(rr_true[s2] > A.rtol2 * bb[s2]) || bb[s2] == 0.0;
            // the inner FP32 iterations run on r scaled by a power of two to an
            // RMS near 1 (exact), so that their products stay far from underflow
            int e = 0;
            if (rr_true[s2] > 0.0) frexp(sqrt(rr_true[s2] / ndof), &e);
            scale[s2] = ldexp(1.0, -e);
            unscale[s2] = ldexp(1.0, e);
        }
        const bool more = !(conv[0] && conv[1]) && outer < A.max_outer;
        double u[4] = {0, 0, 0, 0};   // r.z (2), r.r (2) of the preconditioned residual
        if (more)   // scale r, and the first smoothing step of the preconditioner
            for (int tile = lb; tile < L0.ntiles; tile += nblk) {
                const TileNode n = tile_node(L0, ln0, tile);
                if (!n.ok) continue;
                float rv[6], zv[6];
                ld6(Sr + (size_t)n.a * 6, rv);
#pragma unroll
                for (int k = 0; k < 6; ++k) rv[k] *= (float)scale[k / 3];
                st6(Sr + (size_t)n.a * 6, rv);
                dinv_apply(sDi, n.cls, om, rv, zv);
                st6(Sz + (size_t)n.a * 6, zv);
                if (gdepth == 0) {
                    u[0] += (double)dot3(rv, zv);
                    u[1] += (double)dot3(rv + 3, zv + 3);
                }
            }
        if (leader) outer_flag[sidx] = more ? 1 + gdepth : 0;
        if (!grid_sync(gbar, A.err)) return;
        int n_more = 0, gmax = 0;
        flag_stats(outer_flag, A.S, sh, &n_more, &gmax);
        const int Gd = gmax > 0 ? gmax - 1 : 0;   // V-cycle depth of the solves still refining
        if (n_more == 0) {
            for (int s2 = 0; s2 < 2; ++s2)
                if (bb[s2] == 0.0)
                    for (int tile = lb; tile < L0.ntiles; tile += nblk) {
                        const TileNode n = tile_node(L0, ln0, tile);
                        if (n.ok)
                            for (int k = 0; k < 3; ++k) Sx[(size_t)n.a * 6 + 3 * s2 + k] = 0.0;
                    }
            break;
        }
        // ---- z = M r, r.z ----
        if (Gd > 0 && !vcycle_rest(S, lb, more && gdepth > 0, Gd, gbar, A.err, sS, sDi, sv32, sLev, u)) return;
        block_sum<4>(u, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 4; ++k) partB[blockIdx.x * 8 + k] = u[k];
        if (!grid_sync(gbar, A.err)) return;
        double t4[4];
        range_total<4>(partB, blk0, nblk, t4, sh);
        double rz[2] = {t4[0], t4[1]};
        // gain four digits per refinement step, but never solve below a tenth
        // of the final tolerance (in the scaled units of the inner iterations)
        double target[2];
        for (int s2 = 0; s2 < 2; ++s2)
            target[s2] = fmax(A.in_rtol2 * rr_true[s2], 0.01 * A.rtol2 * bb[s2]) * scale[s2] * scale[s2];
        bool ic[2] = {conv[0] || !more, conv[1] || !more};
        float beta[2] = {0.f, 0.f};
        float *pold = S.p0, *pnew = S.p1;
        for (int it = 0; it < A.max_inner; ++it) {
            const bool act = !(ic[0] && ic[1]);
            // ---- p = z + beta p_old, q = K p, p.q ----
            double w[2] = {0, 0};
            if (act) {
                for (int tile = lb; tile < L0.ntiles; tile += nblk) {
                    const TileNode n = tile_node(L0, ln0, tile);
                    __syncthreads();
                    stage_f(L0, ln0, n, Sz, it ? pold : nullptr, beta, sv32);
                    __syncthreads();
                    if (n.ok) {
                        float kq[6], pn[6];
                        stencil_f(sS, sv32, ln0.hc, ln0.hx, ln0.hxy, n.cls, kq);
                        const float *own = sv32 + ln0.hc * 6;
#pragma unroll
                        for (int k = 0; k < 6; ++k) pn[k] = own[k];
                        st6(pnew + (size_t)n.a * 6, pn);
                        st6(Sq + (size_t)n.a * 6, kq);
                        w[0] += (double)dot3(pn, kq);
                        w[1] += (double)dot3(pn + 3, kq + 3);
                    }
                }
            }
            block_sum<2>(w, sh);
            if (threadIdx.x == 0) {
                partA[blockIdx.x * 8 + 0] = w[0];
                partA[blockIdx.x * 8 + 1] = w[1];
                partA[blockIdx.x * 8 + 6] = act ? (double)gdepth : 0.0;
                partA[blockIdx.x * 8 + 7] = act ? 1.0 : 0.0;
            }
            if (!grid_sync(gbar, A.err)) return;
            double pq[2];
            int Gi = 0;   // V-cycle depth of the solves still iterating
            // lagged stop: every block published its solve's activity before the barrier
            if (seg_totals<2>(partA, (int)G, blk0, nblk, pq, sh, &Gi) == 0.0) break;
            float alpha[2];
            for (int s2 = 0; s2 < 2; ++s2) alpha[s2] = (ic[s2] || !(pq[s2] > 0.0)) ? 0.f : (float)(rz[s2] / pq[s2]);
            // ---- d += alpha p, r -= alpha q, first smoothing step z = omega D^-1 r ----
            double u2[4] = {0, 0, 0, 0};
            if (act) {
                for (int tile = lb; tile < L0.ntiles; tile += nblk) {
                    const TileNode n = tile_node(L0, ln0, tile);
                    if (!n.ok) continue;
                    const size_t a = n.a;
                    float pv[6], dv[6], rv[6], qv[6], zv[6];
                    ld6(pnew + a * 6, pv);
                    ld6(Sd + a * 6, dv);
                    ld6(Sr + a * 6, rv);
                    ld6(Sq + a * 6, qv);
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        dv[k] = fmaf(alpha[k / 3], pv[k], dv[k]);
                        rv[k] = fmaf(-alpha[k / 3], qv[k], rv[k]);
                    }
                    dinv_apply(sDi, n.cls, om, rv, zv);
                    st6(Sd + a * 6, dv);
                    st6(Sr + a * 6, rv);
                    st6(Sz + a * 6, zv);
                    if (gdepth == 0) {
                        u2[0] += (double)dot3(rv, zv);
                        u2[1] += (double)dot3(rv + 3, zv + 3);
                        u2[2] += (double)dot3(rv, rv);
                        u2[3] += (double)dot3(rv + 3, rv + 3);
                    }
                }
            }
            // ---- rest of the V-cycle: z = M r, with r.z and r.r ----
            if (Gi > 0) {
                if (!grid_sync(gbar, A.err)) return;
                if (!vcycle_rest(S, lb, act && gdepth > 0, Gi, gbar, A.err, sS, sDi, sv32, sLev, u2)) return;
            }
            block_sum<4>(u2, sh);
            if (threadIdx.x == 0)
                for (int k = 0; k < 4; ++k) partB[blockIdx.x * 8 + k] = u2[k];
            if (!grid_sync(gbar, A.err)) return;
            range_total<4>(partB, blk0, nblk, t4, sh);
            for (int s2 = 0; s2 < 2; ++s2) {
                if (!ic[s2]) {
                    beta[s2] = (rz[s2] != 0.0) ? (float)(t4[s2] / rz[s2]) : 0.f;
                    rz[s2] = t4[s2];
                    ic[s2] = !(t4[2 + s2] > target[s2]) || !(pq[s2] > 0.0);
                } else {
                    beta[s2] = 0.f;
                }
            }
            if (act) ++inner_count;
            float *t = pold;
            pold = pnew;
            pnew = t;
        }
        // ---- x += d (back in the units of x) ----
        for (int tile = lb; tile < L0.ntiles; tile += nblk) {
            const TileNode n = tile_node(L0, ln0, tile);
            if (!n.ok) continue;
#pragma unroll
            for (int k = 0; k < 6; ++k)
                Sx[(size_t)n.a * 6 + k] += (double)Sd[(size_t)n.a * 6 + k] * unscale[k / 3];
        }
        if (!grid_sync(gbar, A.err)) return;
    }
    if (leader) A.it_out[sidx] = inner_count;
}

// f_d of every query of a solve (Eq. 11): f_near where the distance after
// P_C is at most thr, f_far elsewhere; the parameter comes from device memory
// (a captured step reads this step's values) or by value
__global__ void k_fill_fd(float *p, int64_t n, const FdParam *pd, FdParam hp, const double *dpc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const FdParam v = pd ? *pd : hp;
    p[i] = (v.thr >= 0.f && dpc[i] <= (double)v.thr) ? v.f_near : v.f_far;
}

}  // namespace

dd_status dd_fill_fd(dd_ctx *ctx, float *p, int64_t n, const FdParam *pd, FdParam hp, const double *dpc,
                     cudaStream_t s) {
    ctx->launches++;
    k_fill_fd<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, pd, hp, dpc);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

// Tile shape for a level of a solve that gets nblk blocks: fewest estimated
// cycles for the passes over its tiles (a halo round per 256 staged nodes,
// the stencil per warp, the per-node update).
static void pick_tiles(int nx, int ny, int nz, int nblk, Level &L) {
    const int n1[3] = {nx + 1, ny + 1, nz};   // nz: the layers of free nodes
    double best = 1e300;
    for (int tx = 1; tx <= std::min(n1[0], kTileMax); ++tx)
        for (int ty = 1; ty <= std::min(n1[1], kTileMax); ++ty)
            for (int tz = 1; tz <= std::min(n1[2], kTileMax); ++tz) {
                const int T = tx * ty * tz;
                if (T > kBThreads) break;
                const int halo = (tx + 2) * (ty + 2) * (tz + 2);
                if (halo > kHaloMax) continue;
                const int64_t nt = (int64_t)((n1[0] + tx - 1) / tx) * ((n1[1] + ty - 1) / ty) * ((n1[2] + tz - 1) / tz);
                const int64_t passes = (nt + nblk - 1) / nblk;
                const double cost = (double)passes * (700.0 * ((halo + kBThreads - 1) / kBThreads) +
                                                      200.0 * ((T + 31) / 32) + 700.0);
                if (cost < best) {
                    best = cost;
                    L.tx = tx;
                    L.ty = ty;
                    L.tz = tz;
                    L.ntx = (n1[0] + tx - 1) / tx;
                    L.nty = (n1[1] + ty - 1) / ty;
                    L.ntiles = (int)nt;
                }
            }
}

static size_t r256(size_t b) { return (b + 255) / 256 * 256; }

// Launch tables of one CG launch over n solves (built on the host).
struct CGTables {
    std::vector<SegCG> seg;
    std::vector<int> blk_seg;
    int n = 0, total = 0;
    int G = 1;                   // largest number of grid levels
};

// Where those tables and the launch's scratch live on the device.
struct CGDev {
    SegCG *seg = nullptr;
    int *blk_seg = nullptr;
    double *part = nullptr;
    int *flags = nullptr;
    int *it = nullptr;           // [n] inner iterations of every solve (output)
    unsigned *bar = nullptr;
};

static size_t cg_dev_bytes(const CGTables &T) {
    return r256(T.n * sizeof(SegCG)) + r256(T.total * sizeof(int)) + r256((size_t)2 * T.total * 8 * 8) +
           2 * r256((size_t)T.n * sizeof(int)) + 256;
}

static CGDev cg_carve(const CGTables &T, void *base) {
    char *c = (char *)base;
    CGDev D;
    D.seg = (SegCG *)c;
    c += r256(T.n * sizeof(SegCG));
    D.blk_seg = (int *)c;
    c += r256(T.total * sizeof(int));
    D.part = (double *)c;
    c += r256((size_t)2 * T.total * 8 * 8);
    D.flags = (int *)c;
    c += r256((size_t)T.n * sizeof(int));
    D.it = (int *)c;
    c += r256((size_t)T.n * sizeof(int));
    D.bar = (unsigned *)c;
    return D;
}

static dd_status cg_tables(dd_ctx *ctx, const MeshDev *const *gs, const CGBuffers *const *cbs, int n, CGTables &T) {
    int64_t nodes = 0;
    for (int i = 0; i < n; ++i) nodes += gs[i]->n_nodes;
    DD_TRY_CUDA(ctx, cudaFuncSetAttribute((const void *)k_cg_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kDynSmem));
    int occ = 0;
    DD_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_batch, kBThreads, kDynSmem));
    if (occ < 1) return dd_fail(ctx, DD_ERR_CUDA, "CG kernel cannot be resident");
    const int cap = ctx->n_sm;   // one block per SM: fewer barrier arrivals
    if (n > cap) return dd_fail(ctx, DD_ERR_ARG, "more solves than resident CG blocks");
    T.n = n;
    T.G = 1;
    T.seg.assign(n, SegCG{});
    std::vector<int> nblk(n);
    int total = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t share = std::max<int64_t>(1, (int64_t)((double)cap * (double)gs[i]->n_nodes / (double)nodes));
        pick_tiles(gs[i]->nx, gs[i]->ny, gs[i]->nz - cbs[i]->top, (int)share, T.seg[i].lv[0]);
        nblk[i] = (int)std::min<int64_t>(share, T.seg[i].lv[0].ntiles);
        total += nblk[i];
    }
    while (total > cap) {   // trim the largest shares until the grid is co-resident
        int k = (int)(std::max_element(nblk.begin(), nblk.end()) - nblk.begin());
        if (nblk[k] <= 1) return dd_fail(ctx, DD_ERR_ARG, "cannot fit the CG grid");
        --nblk[k];
        --total;
    }
    T.total = total;
    T.blk_seg.assign(total, 0);
    int b0 = 0;
    for (int i = 0; i < n; ++i) {
        const CGBuffers &cb = *cbs[i];
        const size_t n6 = (size_t)gs[i]->n_nodes * 6;
        SegCG &S = T.seg[i];
        S.St64 = cb.St64;
        S.St32 = cb.St32;
        S.b = cb.b;
        S.x = cb.x;
        // the FP64 work arrays hold two FP32 vectors each
        S.r = reinterpret_cast<float *>(cb.r);
        S.d = S.r + n6;
        S.z = reinterpret_cast<float *>(cb.z);
        S.p0 = reinterpret_cast<float *>(cb.p0);
        S.p1 = reinterpret_cast<float *>(cb.p1);
        S.q = reinterpret_cast<float *>(cb.q);
        S.zg = cb.mg_zg;
        S.inv = cb.mg_inv;
        S.ndof = cb.mg_ndof;
        S.blk0 = b0;
        S.nblk = nblk[i];
        S.nlev = cb.nlev;
        S.glev = cb.glev;
        S.omega = (float)cb.omega;
        for (int l = 0; l < cb.nlev; ++l) {
            Level &L = S.lv[l];
            L.nx = cb.lnx[l];
            L.ny = cb.lny[l];
            L.nz = cb.lnz[l];
            L.h = (float)(1 << l);
            L.top = cb.top;
            if (l > 0 && l < cb.glev) pick_tiles(L.nx, L.ny, L.nz - cb.top, S.nblk, L);
            if (l == 0) {
                L.r = S.r;
                L.z = S.z;
                L.t = cb.mg_t0;
            } else if (l < cb.glev) {
                L.r = cb.mg_r[l];
                L.z = cb.mg_z[l];
                L.t = cb.mg_t[l];
            }
        }
        if (cb.glev < cb.nlev && cb.mg_ndof > kMgDirectDofs)
            return dd_fail(ctx, DD_ERR_ARG, "coarsest multigrid level exceeds the direct-solve size");
        T.G = std::max(T.G, cb.glev);
        for (int k = 0; k < nblk[i]; ++k) T.blk_seg[b0 + k] = i;
        b0 += nblk[i];
    }
    return DD_OK;
}

static dd_status cg_upload(dd_ctx *ctx, const CGTables &T, const CGDev &D, cudaStream_t s) {
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(D.seg, T.seg.data(), T.n * sizeof(SegCG), cudaMemcpyHostToDevice, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(D.blk_seg, T.blk_seg.data(), T.total * sizeof(int), cudaMemcpyHostToDevice, s));
    return DD_OK;
}

static dd_status cg_launch(dd_ctx *ctx, const CGTables &T, const CGDev &D, double rtol, int max_it, cudaStream_t s) {
    DD_TRY_CUDA(ctx, cudaMemsetAsync(D.bar, 0, 2 * sizeof(unsigned), s));
    BCGArgs A;
    A.seg = D.seg;
    A.blk_seg = D.blk_seg;
    A.S = T.n;
    A.G = T.G;
    A.part = D.part;
    A.flags = D.flags;
    A.bar = D.bar;
    A.err = ctx->dev_err;
    A.rtol2 = rtol * rtol;
    A.in_rtol2 = 1e-8;                  // each refinement step gains four digits
    A.max_outer = 30;
    A.max_inner = max_it;
    A.it_out = D.it;
    void *args[] = {&A};
    ctx->launches++;
    DD_TRY_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_cg_batch, dim3(T.total), dim3(kBThreads), args,
                                                 kDynSmem, s));
    return DD_OK;
}

// Mixed-precision CG of n systems in one cooperative launch.  *it_dev points
// at the per-system inner iteration counts (device) after the launch.
dd_status dd_cg_segments(dd_ctx *ctx, const MeshDev *const *gs, const CGBuffers *const *cbs, int n, double rtol,
                         int max_it, cudaStream_t s, int **it_dev) {
    CGTables T;
    DD_TRY(cg_tables(ctx, gs, cbs, n, T));
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_BATCH_CG, cg_dev_bytes(T), &w));
    const CGDev D = cg_carve(T, w);
    DD_TRY(cg_upload(ctx, T, D, s));
    DD_TRY(cg_launch(ctx, T, D, rtol, max_it, s));
    *it_dev = D.it;
    return DD_OK;
}

// ---------------------------------------------------------------------------
// One batched DD iteration
// ---------------------------------------------------------------------------
namespace {

// Buffers of one batched step: the concatenated search state, optional
// uploaded CG tables and per-solve f_d (captured form), and the host buffers
// that receive the per-solve statistics.
struct StepIO {
    const CGTables *cgt = nullptr;      // null: built and uploaded per call
    const CGDev *cgd = nullptr;
    double *y_cat = nullptr;
    int32_t *prev_cat = nullptr, *idx_cat = nullptr;
    double *d2_cat = nullptr, *d2nd_cat = nullptr;
    float *fd_cat = nullptr;
    AnnMotion mot{nullptr, nullptr};
    const FdParam *fd_dev = nullptr;    // [n] f_d parameters of every solve in device memory, or null (host values)
    double *h_stats = nullptr;          // [3 n] host copy of (changed, d2 after P_D, d2 after P_C)
    int *h_it = nullptr;                // [n] host copy of the CG iteration counts
    DeferredStats *defer_dev = nullptr, *h_defer = nullptr;
};

size_t concat_bytes(int64_t M) {
    return r256((size_t)M * 96) + 2 * r256((size_t)M * 4) + 2 * r256((size_t)M * 8) + r256((size_t)M * 4) +
           r256((size_t)M * 48) + r256((size_t)M * 4 * kMotStride);
}

void concat_carve(StepIO &io, int64_t M, void *base) {
    char *c = (char *)base;
    io.y_cat = (double *)c;
    c += r256((size_t)M * 96);
    io.prev_cat = (int32_t *)c;
    c += r256((size_t)M * 4);
    io.idx_cat = (int32_t *)c;
    c += r256((size_t)M * 4);
    io.d2_cat = (double *)c;
    c += r256((size_t)M * 8);
    io.d2nd_cat = (double *)c;
    c += r256((size_t)M * 8);
    io.fd_cat = (float *)c;
    c += r256((size_t)M * 4);
    io.mot.q = (float *)c;
    c += r256((size_t)M * 48);
    io.mot.d = (float *)c;
}

// Every device operation of one batched iteration, on stream s and without a
// host synchronisation unless the search needs one (an exact re-search at
// f_d = 1, never in a captured step): per-solve gather and RHS, ONE CG launch,
// per-solve recovery, ONE search over the concatenated states, scatter,
// per-solve statistics and their copy to the host buffers of io.
dd_status enqueue_step(dd_solver **svs, int n, const StepIO &io, const std::vector<FdParam> &fps,
                       dd_search_stats &sst, cudaStream_t s) {
    dd_ctx *ctx = svs[0]->ctx;
    dd_dataset *ds = svs[0]->ds;
    const dd_solve_opts &o0 = svs[0]->o;
    int64_t M = 0;
    for (int i = 0; i < n; ++i) M += svs[i]->g.n_gp;
    cudaEvent_t *ev = svs[0]->ev;   // batch-level phase events
    DD_TRY_CUDA(ctx, dd_event_record(ctx, ev[0], s));
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        DD_TRY(fem_gather_star(ds, sv->cur, sv->g.n_gp, sv->star, sv->ce, s));
        DD_TRY(fem_assemble_rhs(ctx, sv->g, sv->ops, sv->star, sv->ce, sv->f, const_cast<double *>(sv->cb.b), s));
    }
    // ---- one cooperative CG launch for every solve ----
    int *it_dev = nullptr;
    if (o0.cg_mode == 1) {
        for (int i = 0; i < n; ++i) DD_TRY(fem_cg(ctx, svs[i]->g, svs[i]->cb, o0.cg_rtol, o0.cg_max_iter, s));
    } else if (io.cgt) {
        DD_TRY(cg_launch(ctx, *io.cgt, *io.cgd, o0.cg_rtol, o0.cg_max_iter, s));
        it_dev = io.cgd->it;
    } else {
        std::vector<const MeshDev *> gs(n);
        std::vector<const CGBuffers *> cbs(n);
        for (int i = 0; i < n; ++i) {
            gs[i] = &svs[i]->g;
            cbs[i] = &svs[i]->cb;
        }
        DD_TRY(dd_cg_segments(ctx, gs.data(), cbs.data(), n, o0.cg_rtol, o0.cg_max_iter, s, &it_dev));
    }
    DD_TRY_CUDA(ctx, dd_event_record(ctx, ev[1], s));
    for (int i = 0; i < n; ++i) DD_TRY(fem_recover(ds, svs[i]->g, svs[i]->ops, svs[i]->cb.x, svs[i]->star, svs[i]->y,
                                                   svs[i]->dpc, s));
    DD_TRY_CUDA(ctx, dd_event_record(ctx, ev[2], s));

    // ---- one search over the concatenated states ----
    const bool ann = o0.mode == DD_SEARCH_ANN;
    const bool approx = ann || o0.mode == DD_SEARCH_KNNG;   // warm start and motion record
    int64_t off = 0;
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        const int64_t ng = sv->g.n_gp;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.y_cat + off * 12, sv->y, ng * 96, cudaMemcpyDeviceToDevice, s));
        if (approx) {
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.prev_cat + off, sv->cur, ng * 4, cudaMemcpyDeviceToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.mot.q + off * 12, sv->mot.q, ng * 48, cudaMemcpyDeviceToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.mot.d + off * kMotStride, sv->mot.d, ng * 4 * kMotStride, cudaMemcpyDeviceToDevice, s));
        }
        if (ann) {
            ctx->launches++;
            k_fill_fd<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(io.fd_cat + off, ng,
                                                                   io.fd_dev ? io.fd_dev + i : nullptr, fps[i], sv->dpc);
        }
        off += ng;
    }
    SearchOut so{io.idx_cat, io.d2_cat, io.d2nd_cat};
    AnnMotion mot = io.mot;
    if (ann) {
        if (!ds->ann.nlist) return dd_fail(ctx, DD_ERR_STATE, "ANN search needs the partition (ann_nlist)");
        DD_TRY(dd_search_ann_motion(ds, io.y_cat, M, fps[0].f_far, io.fd_cat, io.prev_cat, &mot, o0.ann_budget, so,
                                    &sst, s, o0.eq14));
    } else if (o0.mode == DD_SEARCH_KNNG) {
        DD_TRY(dd_search_knng(ds, io.y_cat, M, o0.f_s, io.prev_cat, &mot, so, &sst, s));
    } else {
        DD_TRY(dd_run_search(ds, o0.mode, o0.certify, o0.f_d_final, o0.f_s, o0.ann_budget, nullptr, io.y_cat, M, so,
                             &sst, s));
    }
    off = 0;
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        const int64_t ng = sv->g.n_gp;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->nxt, io.idx_cat + off, ng * 4, cudaMemcpyDeviceToDevice, s));
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->d2, io.d2_cat + off, ng * 8, cudaMemcpyDeviceToDevice, s));
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->d2nd, io.d2nd_cat + off, ng * 8, cudaMemcpyDeviceToDevice, s));
        if (approx) {
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->mot.q, io.mot.q + off * 12, ng * 48, cudaMemcpyDeviceToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->mot.d, io.mot.d + off * kMotStride, ng * 4 * kMotStride, cudaMemcpyDeviceToDevice, s));
        }
        off += ng;
    }
    DD_TRY_CUDA(ctx, dd_event_record(ctx, ev[3], s));
    for (int i = 0; i < n; ++i)
        DD_TRY(fem_iter_stats(ctx, svs[i]->nxt, svs[i]->cur, svs[i]->d2, svs[i]->dpc, svs[i]->g.n_gp, svs[i]->g.w,
                              svs[i]->stats, s));
    for (int i = 0; i < n; ++i)
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.h_stats + (size_t)i * 3, svs[i]->stats, 3 * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
    if (it_dev) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.h_it, it_dev, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    } else {
        for (int i = 0; i < n; ++i)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.h_it + i, svs[i]->cb.it_out, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    if (io.h_defer)
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(io.h_defer, io.defer_dev, sizeof(DeferredStats), cudaMemcpyDeviceToHost, s));
    return DD_OK;
}

// After the step's stream has drained: phase times, deferred search
// counters, and every solve's bookkeeping and stop rule.
void finish_step(dd_solver **svs, int n, const double *hs, const int *its, dd_search_stats sst,
                 const std::vector<double> &fds, const DeferredStats *dfr, bool graph, dd_iter_info *infos) {
    dd_ctx *ctx = svs[0]->ctx;
    cudaEvent_t *ev = svs[0]->ev;
    // (a failed query must not leave a sticky error for the next call)
    auto elapsed = [](cudaEvent_t a, cudaEvent_t b) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        return ms;
    };
    const float t01 = elapsed(ev[0], ev[1]), t12 = elapsed(ev[1], ev[2]), t23 = elapsed(ev[2], ev[3]);
    if (dfr) {
        const int64_t N = svs[0]->ds->N;
        sst.scan_ms += elapsed(ctx->ev_scan[0], ctx->ev_scan[1]);
        sst.uncertified += (int64_t)(dfr->fb + dfr->ann[2]);
        sst.distances += (int64_t)dfr->fb * N + (int64_t)dfr->ann[0] + (int64_t)dfr->ann[3] + (int64_t)dfr->ann[2] * N;
        sst.points += (int64_t)dfr->ann[5] + (int64_t)dfr->ann[2] * N;
        sst.unique_points += dfr->ann[2] ? N : (int64_t)dfr->ann[4];
        sst.skipped += (int64_t)dfr->ann[1];
        sst.moves += (int64_t)dfr->ann[6];
    }
    for (int i = 0; i < n; ++i) {
        dd_search_stats si = sst;   // the shared search is reported to every solve
        dd_solver_account(svs[i], hs + (size_t)i * 3, its[i], t01, t12, t23, si, fds[i], infos ? &infos[i] : nullptr);
        if (infos) infos[i].graph = graph ? 1 : 0;
    }
}

}  // namespace

// A batched step of a fixed list of solves, kept while the same list is
// stepped again: its own device copies of the CG tables and of the
// concatenated search state (no workspace that another call could move),
// pinned host buffers for f_d and the statistics, and the step captured as a
// CUDA graph once per parity of the solves' association buffers.
struct StepPlan {
    std::vector<uint64_t> ids;
    int n = 0;
    CGTables cgt;
    CGDev cgd;
    StepIO io;
    void *dev = nullptr;
    size_t dev_bytes = 0;
    void *pin = nullptr;
    FdParam *fd_host = nullptr;          // pinned [n]
    bool no_graph = false;               // capture failed once: run this list eagerly
    struct Variant {
        std::vector<char> parity;
        cudaGraphExec_t exec = nullptr;
        uint64_t ws_gen = 0;
        int64_t launches = 0;            // kernels in the graph
        dd_search_stats sst;             // search statistics fixed at capture
    };
    std::vector<Variant> var;
};

static void plan_free(dd_ctx *ctx, StepPlan *P) {
    for (auto &v : P->var)
        if (v.exec) cudaGraphExecDestroy(v.exec);
    if (P->dev) dd_free(ctx, P->dev, P->dev_bytes);
    if (P->pin) cudaFreeHost(P->pin);
    delete P;
}

void dd_plans_drop(dd_ctx *ctx, uint64_t id) {
    if (ctx->plans.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    std::vector<StepPlan *> keep;
    for (StepPlan *P : ctx->plans) {
        if (id == 0 || std::find(P->ids.begin(), P->ids.end(), id) != P->ids.end()) plan_free(ctx, P);
        else keep.push_back(P);
    }
    ctx->plans.swap(keep);
    if (id == 0 || std::find(ctx->last_batch.begin(), ctx->last_batch.end(), id) != ctx->last_batch.end())
        ctx->last_batch.clear();
}

static dd_status plan_make(dd_solver **svs, int n, int64_t M, StepPlan **out) {
    dd_ctx *ctx = svs[0]->ctx;
    const bool cg_seg = svs[0]->o.cg_mode != 1;
    StepPlan *P = new StepPlan();
    P->n = n;
    for (int i = 0; i < n; ++i) P->ids.push_back(svs[i]->id);
    auto fail = [&](dd_status st) {
        plan_free(ctx, P);
        return st;
    };
    if (cg_seg) {
        std::vector<const MeshDev *> gs(n);
        std::vector<const CGBuffers *> cbs(n);
        for (int i = 0; i < n; ++i) {
            gs[i] = &svs[i]->g;
            cbs[i] = &svs[i]->cb;
        }
        dd_status st = cg_tables(ctx, gs.data(), cbs.data(), n, P->cgt);
        if (st != DD_OK) return fail(st);
    }
    const size_t b_cg = cg_seg ? r256(cg_dev_bytes(P->cgt)) : 0, b_cat = concat_bytes(M),
                 b_fd = r256((size_t)n * sizeof(FdParam)),
                 b_def = r256(sizeof(DeferredStats));
    P->dev_bytes = b_cg + b_cat + b_fd + b_def;
    dd_status st = dd_alloc(ctx, &P->dev, P->dev_bytes, "batched step plan");
    if (st != DD_OK) {
        P->dev = nullptr;
        return fail(st);
    }
    char *c = (char *)P->dev;
    if (cg_seg) {
        P->cgd = cg_carve(P->cgt, c);
        P->io.cgt = &P->cgt;
        P->io.cgd = &P->cgd;
    }
    concat_carve(P->io, M, c + b_cg);
    FdParam *fd_dev = (FdParam *)(c + b_cg + b_cat);
    P->io.fd_dev = fd_dev;
    P->io.defer_dev = (DeferredStats *)(c + b_cg + b_cat + b_fd);
    const size_t h_stats = r256((size_t)n * 24), h_it = r256((size_t)n * 4), h_fd = r256((size_t)n * sizeof(FdParam));
    if (cudaHostAlloc(&P->pin, h_stats + h_it + h_fd + r256(sizeof(DeferredStats)), cudaHostAllocDefault) !=
        cudaSuccess) {
        P->pin = nullptr;
        return fail(dd_fail(ctx, DD_ERR_OOM, "batched step plan: pinned host buffers"));
    }
    char *h = (char *)P->pin;
    P->io.h_stats = (double *)h;
    P->io.h_it = (int *)(h + h_stats);
    P->fd_host = (FdParam *)(h + h_stats + h_it);
    P->io.h_defer = (DeferredStats *)(h + h_stats + h_it + h_fd);
    cudaStream_t s = ctx->stream;
    if ((cg_seg && (st = cg_upload(ctx, P->cgt, P->cgd, s)) != DD_OK)) return fail(st);
    if (cudaMemsetAsync(P->io.defer_dev, 0, sizeof(DeferredStats), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(dd_fail(ctx, DD_ERR_CUDA, "batched step plan: upload"));
    if (ctx->plans.size() >= 4) {   // keep the four most recent lists
        plan_free(ctx, ctx->plans.front());
        ctx->plans.erase(ctx->plans.begin());
    }
    ctx->plans.push_back(P);
    *out = P;
    return DD_OK;
}

// Capture the step into a graph for the current parity; null when capture is
// not possible (the caller then runs the step eagerly).
static StepPlan::Variant *plan_capture(StepPlan *P, dd_solver **svs, int n, const std::vector<char> &par,
                                       const std::vector<FdParam> &fps) {
    dd_ctx *ctx = svs[0]->ctx;
    cudaStream_t s = ctx->stream;
    StepPlan::Variant v;
    v.parity = par;
    std::memset(&v.sst, 0, sizeof(v.sst));
    const int64_t l0 = ctx->launches;
    const std::string err0 = ctx->err;
    ctx->capturing = true;
    ctx->defer = P->io.defer_dev;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    dd_status st = DD_OK;
    if (e == cudaSuccess) {
        st = enqueue_step(svs, n, P->io, fps, v.sst, s);
        const cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e == cudaSuccess) e = e2;
    }
    ctx->capturing = false;
    ctx->defer = nullptr;
    v.launches = ctx->launches - l0;
    ctx->launches = l0;          // nothing ran yet; every replay adds v.launches
    v.ws_gen = ctx->ws_gen;
    if (e == cudaSuccess && st == DD_OK && g) e = cudaGraphInstantiate(&v.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || st != DD_OK || !v.exec) {
        cudaGetLastError();      // clear the capture error; this list runs eagerly from now on
        ctx->err = err0;
        P->no_graph = true;
        return nullptr;
    }
    P->var.push_back(v);
    return &P->var.back();
}

extern "C" dd_status dd_solvers_step(dd_solver **svs, int n, dd_iter_info *infos) {
    if (!svs || n < 1 || !svs[0]) return DD_ERR_ARG;
    dd_ctx *ctx = svs[0]->ctx;
    dd_dataset *ds = svs[0]->ds;
    const dd_solve_opts &o0 = svs[0]->o;
    int64_t M = 0;
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        if (!sv || sv->ds != ds) return dd_fail(ctx, DD_ERR_ARG, "dd_solvers_step: solvers must share one data set");
        if (sv->done) return dd_fail(ctx, DD_ERR_STATE, "dd_solvers_step: a solve has already finished");
        if (sv->o.mode != o0.mode || sv->o.certify != o0.certify || sv->o.cg_mode != o0.cg_mode ||
            sv->o.f_s != o0.f_s || sv->o.ann_budget != o0.ann_budget || sv->o.eq14 != o0.eq14)
            return dd_fail(ctx, DD_ERR_ARG,
                           "dd_solvers_step: solvers must share search mode, certify, cg_mode, f_s, ann_budget and eq14");
        for (int j = 0; j < i; ++j)
            if (svs[j] == sv) return dd_fail(ctx, DD_ERR_ARG, "dd_solvers_step: a solver appears twice");
        M += sv->g.n_gp;
    }
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const bool ann = o0.mode == DD_SEARCH_ANN;
    std::vector<double> fds(n);
    std::vector<FdParam> fps(n);
    bool full_fd = false;   // f_d = 1 may need an exact re-search sized on the host
    std::vector<uint64_t> ids(n);
    for (int i = 0; i < n; ++i) {
        ++svs[i]->it;
        fps[i] = dd_solver_fd_param(svs[i], svs[i]->it);
        fds[i] = fps[i].f_far;
        full_fd |= ann && (fps[i].f_far >= 1.0f || (fps[i].thr >= 0.f && fps[i].f_near >= 1.0f));
        ids[i] = svs[i]->id;
    }
    // ---- the same list as the previous step: replay its captured graph ----
    const bool repeat = ids == ctx->last_batch;
    ctx->last_batch = ids;
    StepPlan *P = nullptr;
    if (repeat && !full_fd) {
        for (StepPlan *q : ctx->plans)
            if (q->ids == ids) P = q;
        if (!P) {
            const std::string err0 = ctx->err;
            if (plan_make(svs, n, M, &P) != DD_OK) {
                P = nullptr;     // not enough memory for a plan: step eagerly
                ctx->err = err0;
            }
        }
    }
    if (P && !P->no_graph) {
        std::vector<char> par(n);
        for (int i = 0; i < n; ++i) par[i] = svs[i]->cur != svs[i]->idx_a;
        StepPlan::Variant *v = nullptr;
        for (auto it = P->var.begin(); it != P->var.end(); ++it)
            if (it->parity == par) {
                if (it->ws_gen != ctx->ws_gen) {   // a workspace it uses has moved
                    cudaGraphExecDestroy(it->exec);
                    P->var.erase(it);
                } else {
                    v = &*it;
                }
                break;
            }
        for (int i = 0; i < n; ++i) P->fd_host[i] = fps[i];
        if (!v) v = plan_capture(P, svs, n, par, fps);
        if (v) {
            // this step's f_d values, read by the graph's fill kernels
            DD_TRY_CUDA(ctx, cudaMemcpyAsync((void *)P->io.fd_dev, P->fd_host, n * sizeof(FdParam),
                                             cudaMemcpyHostToDevice, s));
            ctx->launches += v->launches;
            DD_TRY_CUDA(ctx, cudaGraphLaunch(v->exec, s));
            DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
            DD_TRY(dd_check_device_error(ctx, s, "dd_solvers_step"));
            finish_step(svs, n, P->io.h_stats, P->io.h_it, v->sst, fds, P->io.h_defer, true, infos);
            return DD_OK;
        }
    }
    // ---- eager step ----
    StepIO io;
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_BATCH, concat_bytes(M), &w));
    concat_carve(io, M, w);
    std::vector<double> hs((size_t)n * 3);
    std::vector<int> its(n, 0);
    io.h_stats = hs.data();
    io.h_it = its.data();
    dd_search_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    DD_TRY(enqueue_step(svs, n, io, fps, sst, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    DD_TRY(dd_check_device_error(ctx, s, "dd_solvers_step"));
    finish_step(svs, n, hs.data(), its.data(), sst, fds, nullptr, false, infos);
    return DD_OK;
}

extern "C" dd_status dd_solve_batch(dd_dataset *ds, int nsolves, const dd_mesh *meshes, const dd_load *loads,
                                    const dd_solve_opts *opts, dd_result *outs) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    if (nsolves < 1 || !meshes || !loads || !outs) return dd_fail(ctx, DD_ERR_ARG, "dd_solve_batch: bad argument");
    std::vector<dd_solver *> svs(nsolves, nullptr);
    dd_status st = DD_OK;
    for (int i = 0; i < nsolves && st == DD_OK; ++i) {
        std::memset(&outs[i], 0, sizeof(dd_result));
        st = dd_solver_create(ds, &meshes[i], &loads[i], opts, &svs[i]);
    }
    while (st == DD_OK) {
        std::vector<dd_solver *> act;
        for (auto *sv : svs)
            if (!sv->done) act.push_back(sv);
        if (act.empty()) break;
        st = dd_solvers_step(act.data(), (int)act.size(), nullptr);
    }
    bool all_conv = true;
    for (int i = 0; i < nsolves && st == DD_OK; ++i) {
        st = dd_solver_result(svs[i], &outs[i]);
        all_conv &= svs[i]->converged;
    }
    for (auto *sv : svs) dd_solver_free(sv);
    if (st == DD_OK && !all_conv) st = DD_ERR_NOT_CONVERGED;
    return st;
}
