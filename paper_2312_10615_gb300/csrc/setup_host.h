// setup_host.h -- host-side set-up arithmetic (dense inverse, Vanka local inverses).
#pragma once
namespace smg {
int dense_inverse(int n, double *A);
int vanka_local_inverse(double h, double eta, double gamma, int cfg, const int *drops, double out[49]);
}  // namespace smg
