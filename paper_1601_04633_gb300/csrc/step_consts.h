// The per-launch constants of the step kernels (dmrt::StepConsts), derived on
// the host from a parameter set and its model constants. One definition,
// used by every entry point that launches a step kernel.
#pragma once
#include "dmrt.h"
#include "lattice.cuh"

namespace dmrt {

// 16-bit thermal storage keeps g_i - w_i theta_ref, w_0 = (1 - a)/5 and
// w_1..4 = (4 + a)/20 (the D2Q5 rest weights of Eq. 42); other storages keep g_i.
inline bool thermal_16bit(int storage) { return storage == DMRT_FP16 || storage == DMRT_BF16; }
inline double thermal_shift0(const dmrt_params& p, const dmrt_consts& k) {
    return thermal_16bit(p.storage) ? (1.0 - k.a) / 5.0 * p.theta_ref : 0.0;
}
inline double thermal_shift1(const dmrt_params& p, const dmrt_consts& k) {
    return thermal_16bit(p.storage) ? (4.0 + k.a) / 20.0 * p.theta_ref : 0.0;
}

// Relaxation rates divided by the squared row norms of M (Eq. 30) and N
// (Eq. 37), the buoyancy scale (Eq. 27), the anti-bounce-back factor (Eq. 45),
// the wall kinds, the thermal storage shifts and the Nusselt scale H / (3 dT)
// of the wall-gradient stencil (Eq. 18).
inline StepConsts make_step_consts(const dmrt_params& p, const dmrt_consts& k) {
    StepConsts s{};
    s.se36 = (float)(k.s_e / 36.0);
    s.snu4 = (float)(k.s_nu / 4.0);
    s.sq12 = (float)(k.s_q / 12.0);
    s.seps36 = (float)(k.s_eps / 36.0);
    s.sk2 = (float)(k.sig_k / 2.0);
    s.se20 = (float)(k.sig_e / 20.0);
    s.snu4t = (float)(k.sig_nu / 4.0);
    s.a = (float)k.a;
    s.gbeta = (float)k.gbeta;
    s.theta_ref = (float)p.theta_ref;
    s.abb = (float)k.abb;
    s.left_fixed = p.left_wall == DMRT_WALL_FIXED;
    s.right_fixed = p.right_wall == DMRT_WALL_FIXED;
    s.gsh0 = (float)thermal_shift0(p, k);
    s.gsh1 = (float)thermal_shift1(p, k);
    s.w0 = (float)((1.0 - k.a) / 5.0);
    s.w1 = (float)((4.0 + k.a) / 20.0);
    const double dT = p.theta_hot - p.theta_cold;
    s.nu_scale = dT != 0.0 ? (double)p.ny / (3.0 * dT) : 0.0;
    return s;
}

}  // namespace dmrt
