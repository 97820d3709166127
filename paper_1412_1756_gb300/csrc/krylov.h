// Inner GMRES of the characteristic-mode solver on the device: Krylov
// vectors, preconditioner application, products and orthogonalisation on
// the GPU, the small Hessenberg least-squares problem on the host.
#pragma once

#include "../../include/mlfma.h"

#include <complex>
#include <string>

namespace mlfma {

class DeviceGmres;

// For plan p (FP32 products).  sai: the sparse approximate inverse in the
// near-field strip layout (leaf order; nnz values) or nullptr for none.
DeviceGmres *device_gmres_create(mlfma_plan_t p, const std::complex<double> *sai, int restart, std::string &err);
void device_gmres_destroy(DeviceGmres *g);

// One restarted, right-preconditioned GMRES run on M d = r (M = Z for
// mode 0, X = Im Z for mode 1) in FP32 arithmetic with FP64 inner products:
// r and d are host vectors in canonical order; iterates until the residual
// norm is <= target or maxit iterations were spent.  Returns the iterations
// used, or -1 on failure (err set).
int device_gmres_run(DeviceGmres *g, int mode, const std::complex<double> *r, std::complex<double> *d,
                     double target, int maxit, std::string &err);

// Block variant for real systems with X = Im Z: the p columns of B advance
// together through one product of p real columns per step, each with its
// own basis and least-squares problem (GMRES restarted every `restart`
// steps, right-preconditioned by the real part of sai, nullptr for none).
class BlockGmres;
BlockGmres *block_gmres_create(mlfma_plan_t p, const std::complex<double> *sai, int restart, int cols,
                               std::string &err);
void block_gmres_destroy(BlockGmres *g);

// X D = B for host blocks B, D [n][cols] (canonical order, row-major) in FP32
// arithmetic with FP64 inner products, starting from D itself when guess is
// non-zero (else from 0), until every column's residual is <= tol ||b_c||
// or maxit steps were spent; conv[c] = 1 for columns that
// got there; relres[c] (may be nullptr) receives each column's final
// ||b - X d|| / ||b||.  Returns the steps used (one product of cols columns
// each, plus one per restart for the true residual), or -1 on failure (err
// set).
int block_gmres_run(BlockGmres *g, const double *B, double *D, int guess, double tol, int maxit, int *conv,
                    double *relres, std::string &err);

// Outer Arnoldi basis of cm_ira_solve on the plan's device (arnoldi_device.cu):
// m + 1 complex FP64 vectors of length n.  Host vectors are canonical-order
// complex; each call returns false with err set on a CUDA failure.
class DeviceArnoldi;
DeviceArnoldi *arnoldi_create(mlfma_plan_t p, int64_t n, int m, std::string &err);
void arnoldi_destroy(DeviceArnoldi *a);
bool arnoldi_set(DeviceArnoldi *a, int j, const std::complex<double> *v, std::string &err);   // V_j = v
bool arnoldi_get(DeviceArnoldi *a, int j, std::complex<double> *v, std::string &err);         // v = V_j
// w orthogonalised against V_0..V_j (classical Gram-Schmidt twice): h[i] += the
// coefficients of both passes, *hn = the remaining norm, V_{j+1} = w / *hn,
// and out (when not null) = V_{j+1}.
bool arnoldi_extend(DeviceArnoldi *a, int j, const std::complex<double> *w, std::complex<double> *h, double *hn,
                    std::complex<double> *out, std::string &err);
// V_c <- sum_{i < rows} coef[i * cols + c] V_i for c < cols (all from the old basis)
bool arnoldi_recombine(DeviceArnoldi *a, int rows, int cols, const std::complex<double> *coef, std::string &err);
// V_j <- V_j / ||V_j||, *nrm = ||V_j||
bool arnoldi_normalise(DeviceArnoldi *a, int j, double *nrm, std::string &err);
// out[c] (host, n values each) = sum_{i < rows} coef[i * cols + c] V_i
bool arnoldi_combine(DeviceArnoldi *a, int rows, int cols, const std::complex<double> *coef, std::complex<double> *out,
                     std::string &err);

}  // namespace mlfma
