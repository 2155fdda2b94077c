// Finite-element operators of the constraint projection P_C (fem.cu).
#pragma once

#include <vector>

#include "dd_internal.cuh"

struct MeshDev {
    int nx, ny, nz;
    int64_t n_nodes, n_el, n_gp;
    double hx, hy, hz;
    double w;            // Gauss weight * det J = hx hy hz / 8
    int top_fixed;       // 1: the face z = lz is a Dirichlet boundary too (prescribed rotation)
};

// Physical shape-function gradients dN[gauss point][local node][x,y,z] of
// the (identical) elements of the box.
struct ElemOps {
    double dN[8][8][3];
};

// Geometric multigrid of the constraint projection: level l + 1 halves the
// element counts of level l (rounding up) and doubles the element size, while
// every count is at least 2.  For even counts the coarse space is nested and
// its stiffness is exactly the Galerkin product; an odd count gives a coarse
// box one fine layer longer (not nested: the coarse operator is the
// rediscretised one, and the V-cycle stays symmetric positive definite).
// The hierarchy stops at the first coarse level with at most kMgDirectDofs
// free degrees of freedom, which is solved exactly (a dense inverse applied
// by one block of the solve); the finer levels run on the whole grid.
constexpr int kMgMaxLev = 8;
constexpr int kMgDirectDofs = 400;

struct CGBuffers {
    const double *Ke, *Minv, *b;
    const double *St64;   // stencil table [27 classes][27 offsets][9] (fem_stencil_table)
    const float *St32;    // the same in FP32, blocks padded to 12 values
    // multigrid hierarchy (fem_mg_plan)
    int top = 0;                               // the top layer of nodes is fixed on every level
    int nlev = 1, glev = 1;                    // levels; levels run by the whole grid (glev < nlev:
                                               // level glev is solved directly)
    int lnx[kMgMaxLev], lny[kMgMaxLev], lnz[kMgMaxLev];
    float *mg_t0 = nullptr;                    // level-0 scratch [nodes x 6]
    float *mg_r[kMgMaxLev], *mg_z[kMgMaxLev], *mg_t[kMgMaxLev];   // grid levels 1 .. glev-1
    float *mg_zg = nullptr;                    // coarse solution (level glev, all nodes)
    float *mg_inv = nullptr;                   // inverse of level glev's K on its free DOFs [ndof x ndof]
    int mg_ndof = 0;
    double omega = 0.5;                        // damped block-Jacobi weight of the smoother
    double *x, *r, *z, *p0, *p1, *q, *part;
    unsigned *bar;
    int *it_out;
    double *res_out;
};

inline MeshDev fem_mesh(const dd_mesh &m) {
    MeshDev g;
    g.nx = m.nx;
    g.ny = m.ny;
    g.nz = m.nz;
    g.n_nodes = (int64_t)(m.nx + 1) * (m.ny + 1) * (m.nz + 1);
    g.n_el = (int64_t)m.nx * m.ny * m.nz;
    g.n_gp = 8 * g.n_el;
    g.hx = m.lx / m.nx;
    g.hy = m.ly / m.ny;
    g.hz = m.lz / m.nz;
    g.w = g.hx * g.hy * g.hz / 8.0;
    g.top_fixed = 0;
    return g;
}

void fem_elem_ops(const MeshDev &g, ElemOps *ops);
void fem_element_stiffness(const MeshDev &g, const ElemOps &ops, const double *C, double *Ke);
void fem_stencil_table(const double *Ke, double *S);
// Levels of the multigrid hierarchy of a box: element counts per level and
// the number of levels run by the whole grid (fills nlev, glev, lnx, lny, lnz).
void fem_mg_plan(const MeshDev &g, CGBuffers &cb);
// Inverse of the stiffness of the directly solved level (cb.glev, when
// cb.glev < cb.nlev) on its free DOFs, from the stencil table; symmetric, FP32.
void fem_mg_coarse_inverse(const CGBuffers &cb, const double *St64, std::vector<float> &inv);
// Largest eigenvalue of D^-1 K (D: the 3x3 diagonal blocks) by power
// iteration on a small box with the same elements, from the stencil table.
double fem_jacobi_lambda_max(const double *St64);
void fem_traction_force(const MeshDev &g, const dd_load &L, double lx, double ly, double *f);
// Prescribed displacement of the top face turned by theta about the vertical
// axis through its centre, written into the u part of x [n_nodes x 6]
// (the other entries untouched).
void fem_top_rotation(const MeshDev &g, double theta, double lx, double ly, double *x);

dd_status fem_gather_star(dd_dataset *ds, const int32_t *idx, int64_t n_gp, double *star, double *ce,
                          cudaStream_t s);
dd_status fem_assemble_rhs(dd_ctx *ctx, const MeshDev &g, const ElemOps &ops, const double *star,
                           const double *ce, const double *f, double *b, cudaStream_t s);
dd_status fem_block_jacobi(dd_ctx *ctx, const MeshDev &g, const double *Ke, double *Minv, cudaStream_t s);
dd_status fem_cg(dd_ctx *ctx, const MeshDev &g, const CGBuffers &B, double rtol, int max_it,
                 cudaStream_t s);
dd_status fem_cg_mixed(dd_ctx *ctx, const MeshDev &g, const CGBuffers &B, double rtol, int max_it,
                       cudaStream_t s);
dd_status dd_cg_segments(dd_ctx *ctx, const MeshDev *const *gs, const CGBuffers *const *cbs, int n, double rtol,
                         int max_it, cudaStream_t s, int **it_dev);
dd_status fem_recover(dd_dataset *ds, const MeshDev &g, const ElemOps &ops, const double *x,
                      const double *star, double *y, double *dpc, cudaStream_t s);
// out must hold kIterStatsDoubles doubles, zeroed once before the first call.
constexpr int kIterStatsDoubles = 8 + 3 * 256;
dd_status fem_iter_stats(dd_ctx *ctx, const int32_t *idx_new, const int32_t *idx_old, const double *d2,
                         const double *dpc, int64_t n, double w, double *out, cudaStream_t s);
