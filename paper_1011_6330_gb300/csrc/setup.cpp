// Host-side set-up of a tube: unit conversion (Sec. 3), the rho_GJ profile
// (Eq. 5, Eq. 6-7), the empty-tube Poisson problem (Eq. 4) and, for the
// adjoint, its transpose and the profile's analytic derivatives in (B, P, R).
#include <cmath>
#include <cstring>
#include <vector>

#include "sclf_internal.h"

namespace sclf {

namespace {
// cgs constants (CODATA 2018).
constexpr double kC = 2.99792458e10;          // speed of light [cm/s]
constexpr double kE = 4.80320471e-10;         // elementary charge [esu]
constexpr double kMe = 9.1093837015e-28;      // electron mass [g]
constexpr double kG = 6.67430e-8;             // gravitational constant
constexpr double kPi = 3.14159265358979323846;

// rho_GJ / (-(Lambda0^2 / 4 pi)) at dimensionless radius eta = r / R_*.
// Flat (Eq. 5): cos i + 3/2 sqrt(eta) theta_* sin i   (cos(phi) = 1, the
// (R_* / r)^3 factor dropped for the constant-radius tube).
// Frame dragging (Eq. 6 with omega / Omega = kappa / eta^3 from Eq. 7):
//   (f / f1) / alpha [(1 - kappa/eta^3) cos i + 3/2 sqrt(eta) (H / sqrt(f)) theta_* sin i]
// or, for SCLF_GR_BOTH (Omega -> Omega - omega on the prefactor),
//   (f / f1) / alpha (1 - kappa/eta^3) [cos i + 3/2 sqrt(eta) (H / sqrt(f)) theta_* sin i],
// with f, H the curved-space factors at this node (1 without tables), f1 = f
// at the base and alpha = sqrt(1 - r_g / r) when gr_alpha is set.
double shape(const tube_params* p, const tube_derived* d, double eta, double f, double f1,
             double H) {
    if (p->rho_gj_mode != SCLF_RHO_GR)
        return std::cos(p->incl_rad) + 1.5 * std::sqrt(eta) * d->theta_star * std::sin(p->incl_rad);
    const double sin_term =
        1.5 * std::sqrt(eta) * (H / std::sqrt(f)) * d->theta_star * std::sin(p->incl_rad);
    const double drag = 1.0 - d->kappa / (eta * eta * eta);
    const double bracket = p->gr_variant == SCLF_GR_BOTH ? drag * (std::cos(p->incl_rad) + sin_term)
                                                          : drag * std::cos(p->incl_rad) + sin_term;
    double alpha = 1.0;
    if (p->gr_alpha) {
        const double rg_over_rstar = 2.0 * kG * p->mass_g / (kC * kC) / p->Rstar_cm;
        alpha = std::sqrt(1.0 - rg_over_rstar / eta);
    }
    return (f / f1) / alpha * bracket;
}
}  // namespace

int derive(const tube_params* p, tube_derived* d) {
    if (!p || !d) return SCLF_EINVAL;
    std::memset(d, 0, sizeof(*d));
    if (!(p->Nz >= 2 && p->Nz <= (int64_t(1) << 24))) return SCLF_EINVAL;
    if (!(p->L_over_R > 0.0) || !std::isfinite(p->L_over_R)) return SCLF_EINVAL;
    if (p->precision != SCLF_FP32 && p->precision != SCLF_FP64 && p->precision != SCLF_FIX32)
        return SCLF_EINVAL;
    if (p->precision == SCLF_FIX32 && p->accumulate != SCLF_ACC_FIXED64) return SCLF_EINVAL;
    if (p->precision == SCLF_FIX32 && p->Nz < 16) return SCLF_EINVAL;   // per-thread runs fit int32
    if (p->accumulate != SCLF_ACC_FIXED64 && p->accumulate != SCLF_ACC_FP64) return SCLF_EINVAL;
    if (p->rho_gj_mode < SCLF_RHO_FLAT || p->rho_gj_mode > SCLF_RHO_USER) return SCLF_EINVAL;
    if (p->rho_gj_mode == SCLF_RHO_USER && !p->rho_gj_user) return SCLF_EINVAL;
    if (!(p->capacity >= 0 && p->capacity <= (int64_t(1) << 31) - kMaxTile)) return SCLF_EINVAL;
    if (p->compact_interval < 0) return SCLF_EINVAL;
    if (p->sort_interval < 0) return SCLF_EINVAL;
    if (p->push_stages < 0 || p->push_stages > kMaxPushStages) return SCLF_EINVAL;
    if (p->launch_overlap < -1 || p->launch_overlap > 1) return SCLF_EINVAL;
    if (p->gr_variant != SCLF_GR_COS && p->gr_variant != SCLF_GR_BOTH) return SCLF_EINVAL;
    if (p->gr_alpha != 0 && p->gr_alpha != 1) return SCLF_EINVAL;
    if (p->rho_gj_mode == SCLF_RHO_GR) {
        for (int64_t j = 0; j <= p->Nz; ++j) {
            if (p->gr_f && !(std::isfinite(p->gr_f[j]) && p->gr_f[j] > 0.0)) return SCLF_EINVAL;
            if (p->gr_H && !std::isfinite(p->gr_H[j])) return SCLF_EINVAL;
        }
        if (p->gr_alpha && !(2.0 * kG * p->mass_g / (kC * kC) < p->Rstar_cm)) return SCLF_EINVAL;
    }

    if (p->rho_gj_mode == SCLF_RHO_GR && !(p->P_s > 0.0 && p->Rstar_cm > 0.0 && p->mass_g >= 0.0))
        return SCLF_EINVAL;
    // Sec. 3: Omega, theta_p = sqrt(Omega R_* / c), R_p = R_* theta_p,
    // n_GJ = Omega B cos i / (2 pi c e), omega_p = sqrt(4 pi n e^2 / m).
    if (p->P_s > 0.0 && p->Rstar_cm > 0.0) {
        d->Omega = 2.0 * kPi / p->P_s;
        d->theta_p = std::sqrt(d->Omega * p->Rstar_cm / kC);
        d->R_cm = p->R_cm > 0.0 ? p->R_cm : p->Rstar_cm * d->theta_p;
        d->n0 = d->Omega * p->B_G / (2.0 * kPi * kC * kE);
        d->omega_p0 = std::sqrt(4.0 * kPi * d->n0 * kE * kE / kMe);
        d->Lambda0 = d->omega_p0 * d->R_cm / kC;
        const double rg = 2.0 * kG * p->mass_g / (kC * kC);
        d->kappa = 0.4 * rg / p->Rstar_cm;                  // Eq. 7
        d->theta_star = 0.67 * d->theta_p;                  // Eq. 5 text
        d->R_over_Rstar = d->R_cm / p->Rstar_cm;
    }
    if (p->lambda_override > 0.0) d->Lambda0 = p->lambda_override;
    if (p->rho_gj_mode != SCLF_RHO_USER && !(d->Lambda0 > 0.0)) return SCLF_EINVAL;

    d->L = p->L_over_R;
    d->dz = d->L / double(p->Nz);
    if (p->dt > 0.0) {
        d->dt = p->dt;
    } else {
        if (!(d->Lambda0 > 0.0)) return SCLF_EINVAL;
        d->dt = std::fmin(0.4 * d->dz, 0.2 / d->Lambda0);
    }
    if (!(d->dt > 0.0 && d->dt < d->dz)) return SCLF_EINVAL;   // c dt < dz

    if (p->rho_gj_mode == SCLF_RHO_USER) {
        d->rho0 = p->rho_gj_user[0];
    } else {
        const double f0 = p->gr_f ? p->gr_f[0] : 1.0, h0 = p->gr_H ? p->gr_H[0] : 1.0;
        d->rho0 = -(d->Lambda0 * d->Lambda0 / (4.0 * kPi)) * shape(p, d, 1.0, f0, f0, h0);
    }
    if (!std::isfinite(d->rho0)) return SCLF_EINVAL;
    if (p->macro_charge != 0.0) {
        d->s = p->macro_charge;
    } else {
        if (p->target_particles <= 0) return SCLF_EINVAL;
        d->s = -std::fabs(d->rho0) * d->L / double(p->target_particles);
    }
    if (!(d->s < 0.0) || !std::isfinite(d->s)) return SCLF_EINVAL;
    d->pos_unit = p->precision == SCLF_FIX32 ? std::ldexp(1.0, -fix32_bits(p->Nz)) : 1.0;
    return SCLF_OK;
}

int build_rho_gj(const tube_params* p, const tube_derived* d, double* rho) {
    const int64_t nz = p->Nz;
    if (p->rho_gj_mode == SCLF_RHO_USER) {
        for (int64_t j = 0; j <= nz; ++j) {
            if (!std::isfinite(p->rho_gj_user[j])) return SCLF_EINVAL;
            rho[j] = p->rho_gj_user[j];
        }
        return SCLF_OK;
    }
    const double scale = -(d->Lambda0 * d->Lambda0 / (4.0 * kPi));
    const double f1 = p->gr_f ? p->gr_f[0] : 1.0;
    for (int64_t j = 0; j <= nz; ++j) {
        const double z = double(j) * d->dz;                 // in R
        const double eta = 1.0 + z * d->R_over_Rstar;       // r / R_*
        rho[j] = scale * shape(p, d, eta, p->gr_f ? p->gr_f[j] : 1.0, f1,
                               p->gr_H ? p->gr_H[j] : 1.0);
    }
    return SCLF_OK;
}

// Eq. 4 with an empty tube: phi'' - phi / R^2 = 4 pi rho_GJ (R = 1) on the
// nodes, phi_0 = 0 and phi'(L) = 0 through the ghost phi_{Nz+1} = phi_{Nz-1}.
// Tridiagonal in phi_1..phi_Nz; Thomas elimination (the matrix is strictly
// diagonally dominant, |2 + dz^2| > 2, so no pivoting is needed).
void solve_poisson(const double* rho, int64_t nz, double dz, double* phi) {
    const double diag = -(2.0 + dz * dz);
    const double rhs_scale = 4.0 * kPi * dz * dz;
    // forward sweep; cp[i] and dp[i] for unknown i = 1..nz stored at i
    double* cp = new double[nz + 1];
    double* dp = new double[nz + 1];
    for (int64_t i = 1; i <= nz; ++i) {
        const double sub = (i == 1) ? 0.0 : (i == nz ? 2.0 : 1.0);
        const double sup = (i == nz) ? 0.0 : 1.0;
        const double rhs = rhs_scale * rho[i];
        const double denom = diag - (i == 1 ? 0.0 : sub * cp[i - 1]);
        cp[i] = sup / denom;
        dp[i] = (rhs - (i == 1 ? 0.0 : sub * dp[i - 1])) / denom;
    }
    phi[0] = 0.0;
    phi[nz] = dp[nz];
    for (int64_t i = nz - 1; i >= 1; --i) phi[i] = dp[i] - cp[i] * phi[i + 1];
    delete[] cp;
    delete[] dp;
}

// Transpose of solve_poisson. With phi_{1..Nz} = A^-1 (4 pi dz^2 rho_{1..Nz})
// and phi_0 = 0, the source adjoint is lrho_{1..Nz} = 4 pi dz^2 A^-T lphi_{1..Nz},
// lrho_0 = 0. A^T swaps A's off-diagonals: row i of A^T has 1 on the left
// (i > 1) and, on the right, 2 in the row before the last (the ghost entry of
// A's last row) and 1 elsewhere. A is diagonally dominant by rows, so A^T is
// by columns and Thomas elimination without pivoting stays stable.
void solve_poisson_transpose(const double* lphi, int64_t nz, double dz, double* lrho) {
    const double diag = -(2.0 + dz * dz);
    double* cp = new double[nz + 1];
    double* dp = new double[nz + 1];
    for (int64_t i = 1; i <= nz; ++i) {
        const double sub = (i == 1) ? 0.0 : 1.0;
        const double sup = (i == nz) ? 0.0 : (i + 1 == nz ? 2.0 : 1.0);
        const double denom = diag - (i == 1 ? 0.0 : sub * cp[i - 1]);
        cp[i] = sup / denom;
        dp[i] = (lphi[i] - (i == 1 ? 0.0 : sub * dp[i - 1])) / denom;
    }
    double* y = new double[nz + 1];
    y[nz] = dp[nz];
    for (int64_t i = nz - 1; i >= 1; --i) y[i] = dp[i] - cp[i] * y[i + 1];
    const double scale = 4.0 * kPi * dz * dz;
    lrho[0] = 0.0;
    for (int64_t i = 1; i <= nz; ++i) lrho[i] = scale * y[i];
    delete[] cp;
    delete[] dp;
    delete[] y;
}

// shape() and its derivatives in eta and theta_* at one node, written out
// from the same closed forms (Eq. 5, Eq. 6-7):
//   flat: d/deta = (3/4) theta_* sin i / sqrt(eta), d/dtheta_* = (3/2) sqrt(eta) sin i;
//   frame dragging: with T = (3/2) sqrt(eta) (H / sqrt f) theta_* sin i,
//   D = 1 - kappa / eta^3 (dD/deta = 3 kappa / eta^4) and
//   alpha = sqrt(1 - r_g / (R_* eta)) (dalpha/deta = (r_g / R_*) / (2 alpha eta^2)),
//   the bracket's derivatives by the product rule, then (f / f1) / alpha.
namespace {
struct ShapeD {
    double s, d_eta, d_theta;
};
ShapeD shape_d(const tube_params* p, const tube_derived* d, double eta, double f, double f1,
               double H) {
    const double ci = std::cos(p->incl_rad), si = std::sin(p->incl_rad);
    const double se = std::sqrt(eta), th = d->theta_star;
    if (p->rho_gj_mode != SCLF_RHO_GR)
        return {ci + 1.5 * se * th * si, 0.75 * th * si / se, 1.5 * se * si};
    const double hs = H / std::sqrt(f);
    const double t = 1.5 * se * hs * th * si;
    const double t_eta = 0.75 * hs * th * si / se;
    const double t_th = 1.5 * se * hs * si;
    const double e3 = eta * eta * eta;
    const double drag = 1.0 - d->kappa / e3;
    const double drag_eta = 3.0 * d->kappa / (e3 * eta);
    double b, b_eta, b_th;
    if (p->gr_variant == SCLF_GR_BOTH) {
        b = drag * (ci + t);
        b_eta = drag_eta * (ci + t) + drag * t_eta;
        b_th = drag * t_th;
    } else {
        b = drag * ci + t;
        b_eta = drag_eta * ci + t_eta;
        b_th = t_th;
    }
    double a = 1.0, a_eta = 0.0;
    if (p->gr_alpha) {
        const double g = 2.0 * kG * p->mass_g / (kC * kC) / p->Rstar_cm;
        a = std::sqrt(1.0 - g / eta);
        a_eta = g / (eta * eta) / (2.0 * a);
    }
    const double w = f / f1;
    return {w * b / a, w * (b_eta / a - b * a_eta / (a * a)), w * b_th / a};
}
}  // namespace

// d/d(B, P, R) of sum_j d_rho_j rho_GJ,j on a fixed grid (z_j = j dz in
// units of R), with the grid, dt and s held at the values of the unperturbed
// parameters and R an independent coordinate (taken at its derived value,
// not R_* theta_p(P)). rho_GJ,j = -(Lambda0^2 / 4 pi) S(eta_j, theta_*) with
// Lambda0^2 = 4 pi n0 e^2 R^2 / (m c^2) proportional to B R^2 / P (Sec. 3;
// held when lambda_override is set), theta_* = 0.67 (Omega R_* / c)^(1/2)
// proportional to P^(-1/2) and eta_j = 1 + z_j R / R_*, so
//   d rho_j / dB = rho_j / B,
//   d rho_j / dP = -rho_j / P - (Lambda0^2 / 4 pi) dS/dtheta_* (-theta_* / 2P),
//   d rho_j / dR = 2 rho_j / R - (Lambda0^2 / 4 pi) dS/deta z_j / R_*,
// the Lambda0 terms dropped when Lambda0 is overridden. The f, H node tables
// belong to the nodes and do not move. A caller-supplied profile does not
// depend on B, P, R: all three are 0.
int rho_gj_parameter_gradient(const tube_params* p, const double* d_rho, double* grad) {
    grad[0] = grad[1] = grad[2] = 0.0;
    if (p->rho_gj_mode == SCLF_RHO_USER) return SCLF_OK;
    tube_derived d0;
    int rc = derive(p, &d0);
    if (rc) return rc;
    tube_params q = *p;
    q.R_cm = d0.R_cm;
    q.dt = d0.dt;
    q.macro_charge = d0.s;
    tube_derived d;
    if ((rc = derive(&q, &d))) return rc;
    const bool lam = !(q.lambda_override > 0.0);
    const double scale = -(d.Lambda0 * d.Lambda0 / (4.0 * kPi));
    const double dth_dP = (q.P_s > 0.0 && q.Rstar_cm > 0.0) ? -d.theta_star / (2.0 * q.P_s) : 0.0;
    const double deta_dR = q.Rstar_cm > 0.0 ? 1.0 / q.Rstar_cm : 0.0;     // times z_j
    const double f1 = q.gr_f ? q.gr_f[0] : 1.0;
    double gB = 0.0, gP = 0.0, gR = 0.0;
    for (int64_t j = 0; j <= q.Nz; ++j) {
        const double z = double(j) * d.dz;
        const double eta = 1.0 + z * d.R_over_Rstar;
        const ShapeD sd = shape_d(&q, &d, eta, q.gr_f ? q.gr_f[j] : 1.0, f1,
                                  q.gr_H ? q.gr_H[j] : 1.0);
        const double rho = scale * sd.s;
        double dB = 0.0, dP = scale * sd.d_theta * dth_dP, dR = scale * sd.d_eta * z * deta_dR;
        if (lam) {
            dB += rho / q.B_G;
            dP -= rho / q.P_s;
            dR += 2.0 * rho / d.R_cm;
        }
        gB += d_rho[j] * dB;
        gP += d_rho[j] * dP;
        gR += d_rho[j] * dR;
    }
    grad[0] = gB;
    grad[1] = gP;
    grad[2] = gR;
    return SCLF_OK;
}

}  // namespace sclf
