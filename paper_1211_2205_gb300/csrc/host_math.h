// Host-side mathematics of the StaRMAP stepper: moment matrices, grid
// assignment, lambda_max, E(c).  FP64, no CUDA.
#pragma once
#include <string>
#include <vector>

namespace starmap {

// One real moment (section 3): R_l^m (imag = false) or I_l^m (imag = true),
// or psi_l for the slab system (m = 0).
struct Moment {
    int l = 0, m = 0;
    bool imag = false;
    int grid = 0;    // 0 = G11, 1 = G21, 2 = G12, 3 = G22
    int local = 0;   // index among the components of its grid
};

struct SystemMatrices {
    int system = 0, N = 0, ncomp = 0;
    std::vector<Moment> moms;
    std::vector<double> Mx, My;     // dense row-major ncomp x ncomp
    double lambda_max = 0.0;
    int grid_count[4] = {0, 0, 0, 0};
};

// Build Mx, My, moment list, grid placement and lambda_max.
// Returns false with a message in err on failure.
bool build_system(int system, int N, SystemMatrices& out, std::string& err);

// Real harmonic of every component (section 3) at the direction with
// cosine mu to the z axis and azimuth phi (the moments of a unit beam).
bool direction_moments(int system, int N, double mu, double phi, std::vector<double>& out, std::string& err);

// E(c) = (exp(c) - 1)/c, section 5.6.
double expm1div(double c);

// Largest |eigenvalue| of a real symmetric matrix given densely (n x n).
double symmetric_spectral_radius(const std::vector<double>& A, int n);

}  // namespace starmap
