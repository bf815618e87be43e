// Internal declarations shared by the library's CUDA translation units.
//
// Device data layout: every level-l field is (N_l+1) x (N_l+1) nodes stored
// row-major with a row pitch P_l (elements, a multiple of 32) so that each row
// starts on a 256-byte boundary; element (i, j) is at j*P_l + i, with i the x
// index and j the y index (j = N_l is the lid).
//
// The multigrid works in a scaled form.  With kappa = 3/10 for the compact
// operator and 1/4 for the 5-point operator, the stored right-hand side is
// g = -kappa h^2 f, the Gauss-Seidel value of node P is
//     compact:  0.2 * sum(edge neighbours) + 0.05 * sum(diagonal neighbours) + g_P
//     5-point:  0.25 * sum(edge neighbours) + g_P
// (the SOR update of Eq. (15) at beta = 1, divided through by its diagonal),
// the local residual is rho = (Gauss-Seidel value) - psi_P, so that
// f - L_h psi = -rho / (kappa h^2), and full-weighting the fine residual onto
// the coarse grid gives the coarse scaled right-hand side g_c = 4 R(rho).
// Relative residual norms are scale-free: ||rho|| / ||g|| = ||f - L psi|| / ||f||.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace lcx {

constexpr int kLogN = 65536;
constexpr int kMaxLevels = 16;

constexpr int kStatusNoConv = 1;
constexpr int kStatusNonFinite = 2;

// Device-resident solver state, one per context.
struct DevState {
    int cycles;       // V-cycles done in the solve in progress
    int status;       // kStatus* bits, sticky until read by the host
    int last_cycles;  // cycles of the last finished solve
    int pad0;
    double last_rel;  // relative residual at the end of the last solve
    unsigned long long nsolves;
    double mon[3];    // max|d omega|/dt, RES_psi, RES_omega
    double pad1;
    int log[kLogN];   // cycles per solve, ring buffer indexed by nsolves
};

// Coefficients of one SSPRK(5,4) stage in low-storage form.
//   mode 0: out = a0 W0 + a1 in + bdt L
//   mode 1: as mode 0, and acc = acc_in * in
//   mode 2: as mode 0, and acc = acc + acc_in * in + acc_L * L
//   mode 3: out = acc + a1 in + bdt L
struct StageCoef {
    double a0, a1, bdt, acc_in, acc_L;
    int mode;
};

// ---- launchers (lc_kernels.cu); each enqueues on `s` and returns the launch error
template <typename T>
cudaError_t launch_smooth_colour(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int colour, T beta);
template <typename T>
cudaError_t launch_residual_restrict(cudaStream_t s, int op, const T *psi, const T *g, int Nf, int Pf, T *gc,
                                     T *psic, int Pc);
template <typename T>
cudaError_t launch_prolong_correct(cudaStream_t s, T *psi, int Nf, int Pf, const T *ec, int Pc);
template <typename T>
cudaError_t launch_coarsest(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int nsweeps, T beta);
template <typename T>
cudaError_t launch_residual_norm(cudaStream_t s, int op, const T *psi, const T *g, int N, int P, double *partials);

int residual_norm_blocks(int N);
int assemble_blocks(int N);
int monitor_blocks(int N);

cudaError_t launch_assemble_rhs(cudaStream_t s, int op, const double *omega, double *g, int N, int P, double *gpart);
cudaError_t launch_finish_norm(cudaStream_t s, const double *rpart, int nr, const double *gpart, int ng, DevState *ds,
                               cudaGraphConditionalHandle h, double tol, int max_cycles);
cudaError_t launch_thom(cudaStream_t s, const double *psi, double *W0, double *Wa, double *Wb, int N, int P, double U,
                        int profile);
cudaError_t launch_rhs_stage(cudaStream_t s, const double *psi, const double *in, const double *W0, double *acc,
                             double *out, int N, int P, double Re, int advect, StageCoef c);
cudaError_t launch_monitor(cudaStream_t s, const double *psi0, const double *psi1, const double *w0, const double *w1,
                           int N, int P, double *part, DevState *ds, double dt);
cudaError_t launch_zero_walls(cudaStream_t s, double *psi, int N, int P);

// Sets the calling thread's lc_last_error() message.
void set_last_error(const char *msg);

}  // namespace lcx
