// Kernel launchers (host functions defined in the .cu files).
#pragma once

#include "internal.h"

namespace igabem {

// set-up (k_setup.cu)
void launch_gauss_geometry(const DeviceProblem &d, const HostSetup &S, cudaStream_t st);
void launch_node_geometry(const DeviceProblem &d, const HostSetup &S, cudaStream_t st);
void launch_pair_consts(const DeviceProblem &d, const HostSetup &S, double kappa, double eta, cudaStream_t st);
bool m2l_rows_supported(const HostSetup &S, const igabem_options &o, int R);
// stored M2L coupling blocks (m2l_stored): complex entries of level l, and their generation at set-up
size_t m2l_stored_entries(const HostSetup &S, int l);
void launch_m2l_fill(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, cudaStream_t st);
void launch_m2l_rows(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                     bool fp32, cudaStream_t st);
// tensor-core M2L for R right-hand sides (k_m2l_tc.cu); yhat from xhat through d.tc_bimg
bool m2l_tc_supported(const HostSetup &S, int R);
size_t m2l_tc_image_bytes(const HostSetup &S, int l, int R);
void launch_m2l_tc(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st);
// bounded-wait self-test: status[0] = 1 when the wait on an mbarrier nothing arrives at gave up
void launch_wait_selftest(int *status, double limit_s, cudaStream_t st);
// set-up scratch bytes of launch_near_field (element tables of the regular quadrature)
size_t near_table_bytes(const HostSetup &S, const igabem_options &o);
void launch_near_field(const DeviceProblem &d, const HostSetup &S, const igabem_options &o,
                       cudaStream_t st);

// leaf kernels (k_leaf.cu)
bool leaf_kernels_supported(const HostSetup &S);
void launch_near_spmv(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                      cudaStream_t st);
void launch_p2m(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st);
void launch_l2p(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, cudaStream_t st);
// leaf moment matrices for the many-column P2M / L2P (set up once per problem)
bool leaf_moments_supported(const HostSetup &S);
size_t leaf_moment_entries(const HostSetup &S);
void launch_leaf_moments(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, cudaStream_t st);
void launch_block_inverse(const DeviceProblem &d, const HostSetup &S, cudaStream_t st);
void launch_block_apply(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                        cudaStream_t st);
// z = M^-1 r for the block Jacobi preconditioner (k_apply.cu)
void launch_precond(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                    const double *r, double *z, cudaStream_t st);
void launch_blocks_to_fp32(const double *src, float *dst, size_t n, cudaStream_t st);

// operator application (k_apply.cu): y = A x for R columns, x and y device [N][R] complex
void launch_matvec(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                   const double *x, double *y, cudaStream_t st);

// right-hand sides and far field (k_solver.cu)
// kind 0: plane waves with directions dirs; kind 1: point sources at the points dirs
void launch_rhs(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                const double *dirs_dev, double *b, cudaStream_t st, int kind = 0);
// rho[e][q][r] = w_q h^2 sum_k psi_k(q) dens[.][r]: the weighted density at the Gauss points (complex)
void launch_density(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R, const double *dens,
                    double *rho, cudaStream_t st);
// scratch: device space for E ng^2 R complex values (the weighted density at the Gauss points)
void launch_farfield(const DeviceProblem &d, const HostSetup &S, const igabem_options &o, int R,
                     const double *dens, int n_dir, const double *xhat_dev, double *uinf, double *scratch,
                     cudaStream_t st);

// GMRES vector kernels (k_solver.cu); vectors [N][R] complex, per-column results [.][R]
// h[i][r] = sum_n conj(V_i[n][r]) w[n][r] for i < nv (V_i = V + i*N*R)
void launch_multidot(const double *V, int nv, const double *w, long N, int R, double *red,
                     double *h, cudaStream_t st);
// w[n][r] -= sum_i V_i[n][r] h[i][r]
void launch_multiaxpy(const double *V, int nv, const double *h, double *w, long N, int R,
                      cudaStream_t st);
// x[n][r] += sum_i V_i[n][r] y[i][r]
void launch_update(const double *V, int nv, const double *y, double *x, long N, int R,
                   cudaStream_t st);
// nrm[r] = ||w[:, r]||_2
void launch_norms(const double *w, long N, int R, double *red, double *nrm, cudaStream_t st);
// w[n][r] *= s[r] (real), dst may equal w
void launch_scale(const double *w, const double *s, double *dst, long N, int R, cudaStream_t st);
// r = b - y
void launch_sub(const double *b, const double *y, double *r, long n, cudaStream_t st);

// Device-side state of GMRES(m) for R columns (all device memory): the Arnoldi index j of the cycle,
// the rotated Hessenberg matrices, Givens rotations, g, the per-column Krylov dimension, iteration count
// and finished flag.
struct GmDev {
  int m, R, maxit;
  double tol;
  int *j;                     // Arnoldi index
  int *k, *its, *done;        // [R]
  int *flags;                 // [2]: every column finished; non-finite value met
  double2 *H;                 // [(m+1)][m][R]
  double2 *cs, *sn;           // [m][R]
  double2 *g, *y;             // [(m+1)][R]
  double2 *hA, *hB;           // [(m+1)][R]: the two Gram-Schmidt passes
  double *nrm, *s, *bn;       // [R]
  double *V, *w;              // basis [(m+1)][N][R] and the new vector [N][R]
};
// after the matrix-vector product w = A V_j: two CGS passes, the norm, the Arnoldi / Givens update
// (k_gm_arnoldi), V_{j+1} = w / h_{j+1,j}; j advances on the device
void launch_gm_iteration_tail(const GmDev &G, double *red, long N, cudaStream_t st);
// dst = V_j (j read on the device)
void launch_copy_vj(const GmDev &G, double *dst, long N, cudaStream_t st);
// cycle start from beta [R] and the active flags [R] (device)
void launch_gm_init(const GmDev &G, const double *beta, const int *active, cudaStream_t st);
// y = H^-1 g per column
void launch_gm_solve(const GmDev &G, cudaStream_t st);

}  // namespace igabem
