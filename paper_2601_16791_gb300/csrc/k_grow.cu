// k_grow.cu -- radii of the growing planets (arXiv 2601.16791, Sec. 3.3,
// Eqs. 14 and 16), on demand (mx_planets): the step does not use them.  The
// per-step growth update itself runs at the start of each step's first kick
// launch (k_prep, mx_growth.cuh).
#include "mx_common.cuh"
#include "mx_growth.cuh"
#include "mx_kernels.h"

namespace mx {

// One block per system: the radius of every growing big body at t = (global
// step index) x h, from the current state (0 for bodies that do not grow).
__global__ void __launch_bounds__(kThreads) k_radius(Dev d) {
  const SysDev& S = d.sys[blockIdx.x];
  __shared__ double red[3][kThreads];
  double P[3];
  big_momentum(d, S, red, P);
  const double t = (double)d.gstep[0] * S.h;
  for (int i = threadIdx.x; i < S.nbig; i += blockDim.x) {
    const int b = S.boff + i;
    const Growth G = d.grow[b];
    double rad = 0.0;
    if (S.grow_on && G.grows && !removed(d, S.off + i)) {
      double r, v2, R;
      big_rv2(d, S, i, P, &r, &v2, &R);
      const double cs = S.hr1 * pow(R, S.flare) * sqrt(S.mu0 / R);
      if (t <= G.tc) {
        const double mu = S.G * growth_mass(G, t);
        rad = inflated_radius(mu, cs, semimajor_or_r(S.mu0 + mu, r, v2) * cbrt(mu / (3.0 * S.mu0)));
      } else {
        const double muc = S.G * G.mc;
        const double ac = semimajor_or_r(S.mu0 + muc, r, v2);
        rad = inflated_radius(muc, cs, ac * cbrt(muc / (3.0 * S.mu0))) -
              G.dr * (1.0 - exp(-(t - G.tc) / G.tg));
      }
    }
    d.brad[b] = rad;
  }
}

void launch_radius(const Dev& d, cudaStream_t st) { k_radius<<<d.nsys, kThreads, 0, st>>>(d); }

}  // namespace mx
