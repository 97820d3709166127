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

}  // namespace mlfma
