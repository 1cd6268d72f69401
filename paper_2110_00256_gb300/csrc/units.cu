// units.cu -- SI scales of the unit systems a caller may work in (§3.3): the
// library's normalised units, reference-frequency / reference-length
// normalisation of PIC codes, Heaviside-Lorentz natural units with 1 MeV.
// Constants: CODATA 2018 (exact SI values where the 2019 SI fixes them).
#include <cmath>

#include "common.cuh"

namespace {

constexpr double kC = 299792458.0;                 // m/s (exact)
constexpr double kQe = 1.602176634e-19;            // C (exact)
constexpr double kHbar = 1.054571817e-34;          // J s (h exact / 2 pi)
constexpr double kMe = 9.1093837015e-31;           // kg
constexpr double kMeV = 1.602176634e-13;           // J (exact)
constexpr double kPi = 3.141592653589793;

qed_status fill(qed_unit_scales *out, double length, double time, double momentum, double energy, double e_field,
                double b_field)
{
    out->length = length, out->time = time, out->momentum = momentum, out->energy = energy;
    out->e_field = e_field, out->b_field = b_field;
    return QED_OK;
}

}  // namespace

using namespace qed;

extern "C" qed_status qed_units_library(qed_unit_scales *out)
{
    clear_error();
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    const double es = kMe * kMe * kC * kC * kC / (kQe * kHbar);
    return fill(out, kHbar / (kMe * kC), kHbar / (kMe * kC * kC), kMe * kC, kMe * kC * kC, es, es / kC);
}

extern "C" qed_status qed_units_reference_frequency(double omega_r, qed_unit_scales *out)
{
    clear_error();
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    if (!(omega_r > 0.0) || !std::isfinite(omega_r)) QED_FAIL(QED_ERR_INVALID_ARG, "omega_r must be > 0");
    const double e = kMe * kC * omega_r / kQe;
    return fill(out, kC / omega_r, 1.0 / omega_r, kMe * kC, kMe * kC * kC, e, e / kC);
}

extern "C" qed_status qed_units_reference_length(double lambda_r, qed_unit_scales *out)
{
    clear_error();
    if (!(lambda_r > 0.0) || !std::isfinite(lambda_r)) QED_FAIL(QED_ERR_INVALID_ARG, "lambda_r must be > 0");
    return qed_units_reference_frequency(2.0 * kPi * kC / lambda_r, out);
}

extern "C" qed_status qed_units_heaviside_lorentz_mev(qed_unit_scales *out)
{
    clear_error();
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    // a field of 1 MeV^2 exerts q_hl * 1 MeV^2 on a unit charge: with q_e = q_hl
    // (sqrt(4 pi alpha)) that is a force of q_hl MeV / (hbar c / MeV)
    const double qhl = std::sqrt(4.0 * kPi * qed::kAlpha);
    const double length = kHbar * kC / kMeV;
    const double e = qhl * kMeV / (kQe * length);  // V/m of one MeV^2
    return fill(out, length, kHbar / kMeV, kMeV / kC, kMeV, e, e / kC);
}
