// FP64 CPU oracle for the particle-pair distance histogram.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition of what
// the hot path computes.  Only the test suite, the smoke check and the CPU
// baseline leg of the benchmark load it; the product library never does, and
// it shares no code with the CUDA path.
//
// What it computes (Reuter & Koefinger, "CADISHI", Sec. 2):
//   for every unique pair of particles (Alg. 1; single species: inner loop
//   from j = i+1, Sec. 2.2) the distance vector is formed, the minimum image
//   convention of Eq. 5 is applied for periodic boxes, the Euclidean distance
//   r is taken and the bin index kappa = (int) nbins * r / r_max is
//   incremented.  Bins are half open, [kappa dr, (kappa+1) dr) (Eq. 4), and
//   pairs with kappa >= nbins are not counted.
//
// Readings fixed here where the paper is silent (each also listed in the
// design notes):
//   * all arithmetic in IEEE binary64, round to nearest even, no contraction
//     (built with -ffp-contract=off); explicit fma only where written;
//   * coordinates are float32, promoted exactly to binary64 (so d is exact),
//     or binary64 (the distance vector is then rounded once per component);
//   * nint of Eq. 5 is nearbyint (round half to even), as the CPU kernels of
//     the paper use nearbyint (Sec. 4.1);
//   * orthorhombic (Sec. 2.3, diagonal B): k = nearbyint(d * (1/L)),
//     d = fma(-k, L, d) per axis;
//   * triclinic: B is upper triangular with the box vectors as columns;
//     s = B^-1 d by back substitution, k = nearbyint(s), d -= B k, then the
//     minimum of |d + B m|^2 over the 27 shifts m in {-1,0,1}^3 (the
//     neighbouring-cell search of Sec. 2.3 and the three-fold loop over
//     neighbouring boxes of Sec. 4.1);
//   * r^2 = fma(dz,dz, fma(dy,dy, dx*dx)); r = sqrt(r^2);
//     t = (nbins * r) / r_max evaluated left to right (Alg. 1); kappa = floor(t);
//   * histograms for species pairs (a,b), a <= b, in the order
//     (0,0),(0,1),...,(0,S-1),(1,1),...; intra-species pairs i<j only,
//     inter-species pairs all i in a, j in b.
//
// Parity of each function is pinned by the CPU test suite (hand-worked cases,
// pair-count invariant, permutation and translation invariance, the
// ideal-gas closed form, a 125-image brute force for triclinic boxes and an
// exact rational recomputation on tiny inputs).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { BOX_NONE = 0, BOX_ORTHO = 1, BOX_TRICLINIC = 2 };

struct Box {
  int type;
  // row-major 3x3, columns are the box vectors a, b, c (matrix B of Eq. 5)
  double ax, bx, cx, ay, by, cy, az, bz, cz;
  double inv_lx, inv_ly, inv_lz;  // orthorhombic only: 1/L per axis
};

Box make_box(int type, const double* m) {
  Box b;
  b.type = type;
  b.ax = m[0]; b.bx = m[1]; b.cx = m[2];
  b.ay = m[3]; b.by = m[4]; b.cy = m[5];
  b.az = m[6]; b.bz = m[7]; b.cz = m[8];
  b.inv_lx = b.inv_ly = b.inv_lz = 0.0;
  if (type == BOX_ORTHO) {
    b.inv_lx = 1.0 / b.ax;
    b.inv_ly = 1.0 / b.by;
    b.inv_lz = 1.0 / b.cz;
  }
  return b;
}

// Squared length of an explicit vector, in the fixed evaluation order.
inline double norm2(double dx, double dy, double dz) {
  return std::fma(dz, dz, std::fma(dy, dy, dx * dx));
}

// Minimum-image squared distance of the pair (i, j): Alg. 1 steps 1-3 with Eq. 5.
// T is the coordinate type (float or double).
template <typename T>
double pair_r2(const T* xi, const T* xj, const Box& box) {
  // distance vector between the two particles (Alg. 1)
  double dx = (double)xj[0] - (double)xi[0];
  double dy = (double)xj[1] - (double)xi[1];
  double dz = (double)xj[2] - (double)xi[2];
  if (box.type == BOX_ORTHO) {
    // Eq. 5 with diagonal B and B^-1 (Sec. 2.3)
    double kx = std::nearbyint(dx * box.inv_lx);
    double ky = std::nearbyint(dy * box.inv_ly);
    double kz = std::nearbyint(dz * box.inv_lz);
    dx = std::fma(-kx, box.ax, dx);
    dy = std::fma(-ky, box.by, dy);
    dz = std::fma(-kz, box.cz, dz);
  } else if (box.type == BOX_TRICLINIC) {
    // Eq. 5: s = B^-1 d (upper-triangular B: back substitution), d' = d - B nint(s)
    double sz = dz / box.cz;
    double sy = (dy - box.cy * sz) / box.by;
    double sx = (dx - box.bx * sy - box.cx * sz) / box.ax;
    double kx = std::nearbyint(sx);
    double ky = std::nearbyint(sy);
    double kz = std::nearbyint(sz);
    dx = dx - box.ax * kx - box.bx * ky - box.cx * kz;
    dy = dy - box.by * ky - box.cy * kz;
    dz = dz - box.cz * kz;
    // shift to the neighbouring cells and keep the shortest image (Sec. 2.3)
    double best = INFINITY;
    for (int mx = -1; mx <= 1; ++mx)
      for (int my = -1; my <= 1; ++my)
        for (int mz = -1; mz <= 1; ++mz) {
          double ex = dx + box.ax * mx + box.bx * my + box.cx * mz;
          double ey = dy + box.by * my + box.cy * mz;
          double ez = dz + box.cz * mz;
          double r2 = norm2(ex, ey, ez);
          if (r2 < best) best = r2;
        }
    return best;
  }
  return norm2(dx, dy, dz);
}

// Bin index of Alg. 1: (int) nbins * r / r_max, with r = sqrt(r2).  Values at or
// beyond nbins are returned as nbins (not counted).
int64_t bin_of(double r2, double r_max, int32_t nbins) {
  double r = std::sqrt(r2);
  double t = (double)nbins * r;
  t = t / r_max;
  if (!(t < (double)nbins)) return nbins;
  return (int64_t)std::floor(t);
}

inline int64_t hist_index(int64_t a, int64_t b, int64_t S) {
  // position of species pair (a, b), a <= b, in (0,0),(0,1),...,(0,S-1),(1,1),...
  return a * S - a * (a - 1) / 2 + (b - a);
}

// Histogram of one species pair into hist[0..nbins): Alg. 1 (inter) or its
// single-species variant with j > i (intra).
template <typename T>
void histogram_pair(const T* x, int64_t a0, int64_t a1, int64_t b0, int64_t b1, bool intra,
                    const Box& box, double r_max, int32_t nbins, uint64_t* hist, int nthreads) {
  int64_t na = a1 - a0;
  if (na <= 0 || b1 - b0 <= 0) return;
  int nt = nthreads > 0 ? nthreads : 1;
  std::vector<std::vector<uint64_t>> priv(nt, std::vector<uint64_t>((size_t)nbins, 0));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t i = a0; i < a1; ++i) {
#ifdef _OPENMP
    std::vector<uint64_t>& h = priv[(size_t)omp_get_thread_num()];
#else
    std::vector<uint64_t>& h = priv[0];
#endif
    int64_t jstart = intra ? i + 1 : b0;
    for (int64_t j = jstart; j < b1; ++j) {
      double r2 = pair_r2(x + 3 * i, x + 3 * j, box);
      int64_t k = bin_of(r2, r_max, nbins);
      if (k < nbins) h[(size_t)k] += 1;
    }
  }
  for (int t = 0; t < nt; ++t)
    for (int32_t k = 0; k < nbins; ++k) hist[k] += priv[(size_t)t][(size_t)k];
}

// All S(S+1)/2 species-pair histograms of one frame.  Return codes: 0 ok, -1 invalid argument.
template <typename T>
int histogram_all(const T* coords, int64_t n, const int64_t* offsets, int32_t n_species, int32_t box_type,
                  const double* box, double r_max, int32_t nbins, uint64_t* out, int32_t nthreads) {
  if (n < 0 || n_species < 1 || nbins < 1 || !(r_max > 0.0)) return -1;
  if (box_type < BOX_NONE || box_type > BOX_TRICLINIC) return -1;
  if (offsets[0] != 0 || offsets[n_species] != n) return -1;
  for (int32_t s = 0; s < n_species; ++s)
    if (offsets[s + 1] < offsets[s]) return -1;
  double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  Box b = make_box(box_type, box ? box : zero);
  int64_t S = n_species;
  std::memset(out, 0, sizeof(uint64_t) * (size_t)(S * (S + 1) / 2) * (size_t)nbins);
  for (int64_t a = 0; a < S; ++a)
    for (int64_t c = a; c < S; ++c) {
      uint64_t* h = out + hist_index(a, c, S) * nbins;
      histogram_pair(coords, offsets[a], offsets[a + 1], offsets[c], offsets[c + 1], a == c, b,
                     r_max, nbins, h, nthreads);
    }
  return 0;
}

// One species-pair histogram (a <= c) of a frame, the same loops as histogram_all.
template <typename T>
int histogram_one(const T* coords, int64_t n, const int64_t* offsets, int32_t n_species, int32_t a, int32_t c,
                  int32_t box_type, const double* box, double r_max, int32_t nbins, uint64_t* out,
                  int32_t nthreads) {
  if (n < 0 || n_species < 1 || nbins < 1 || !(r_max > 0.0)) return -1;
  if (box_type < BOX_NONE || box_type > BOX_TRICLINIC) return -1;
  if (a < 0 || c < a || c >= n_species) return -1;
  if (offsets[0] != 0 || offsets[n_species] != n) return -1;
  for (int32_t s = 0; s < n_species; ++s)
    if (offsets[s + 1] < offsets[s]) return -1;
  double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  Box b = make_box(box_type, box ? box : zero);
  std::memset(out, 0, sizeof(uint64_t) * (size_t)nbins);
  histogram_pair(coords, offsets[a], offsets[a + 1], offsets[c], offsets[c + 1], a == c, b, r_max, nbins, out,
                 nthreads);
  return 0;
}

}  // namespace

extern "C" {

// the histogram of species pair (a, c), a <= c, alone (float32 coordinates, n x 3)
int dh_oracle_histogram_one(const float* coords, int64_t n, const int64_t* offsets, int32_t n_species, int32_t a,
                            int32_t c, int32_t box_type, const double* box, double r_max, int32_t nbins,
                            uint64_t* out, int32_t nthreads) {
  return histogram_one(coords, n, offsets, n_species, a, c, box_type, box, r_max, nbins, out, nthreads);
}

// float32 coordinates (n x 3)
int dh_oracle_histogram(const float* coords, int64_t n, const int64_t* offsets, int32_t n_species,
                        int32_t box_type, const double* box, double r_max, int32_t nbins,
                        uint64_t* out, int32_t nthreads) {
  return histogram_all(coords, n, offsets, n_species, box_type, box, r_max, nbins, out, nthreads);
}

// binary64 coordinates (n x 3)
int dh_oracle_histogram_f64(const double* coords, int64_t n, const int64_t* offsets, int32_t n_species,
                            int32_t box_type, const double* box, double r_max, int32_t nbins,
                            uint64_t* out, int32_t nthreads) {
  return histogram_all(coords, n, offsets, n_species, box_type, box, r_max, nbins, out, nthreads);
}

double dh_oracle_pair_r2(const float* xi, const float* xj, int32_t box_type, const double* box) {
  double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  Box b = make_box(box_type, box ? box : zero);
  return pair_r2(xi, xj, b);
}

int64_t dh_oracle_bin(double r2, double r_max, int32_t nbins) { return bin_of(r2, r_max, nbins); }

// Batch form of dh_oracle_pair_r2 for m explicit pairs (index arrays).
void dh_oracle_pairs_r2(const float* coords, const int64_t* ii, const int64_t* jj, int64_t m,
                        int32_t box_type, const double* box, double* out) {
  double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  Box b = make_box(box_type, box ? box : zero);
  for (int64_t p = 0; p < m; ++p) out[p] = pair_r2(coords + 3 * ii[p], coords + 3 * jj[p], b);
}

// Radial distribution function of Eq. 1 from histograms of Eqs. 3-4 that hold
// counts summed over n_frames frames: per bin k (r_k = k dr, dr = r_max/nbins,
// Eq. 4), the mean pairs per frame in the bin divided by the pairs a uniform
// pair density N_pairs / V (pair_density[h]) puts in the bin's spherical shell,
// whose volume (4 pi / 3)(r_{k+1}^3 - r_k^3) is the finite-bin form of the
// 4 pi r^2 dr of Eq. 1.  counts and g are n_hist x nbins, row-major.
void dh_oracle_rdf(const uint64_t* counts, int32_t n_hist, int32_t nbins, double r_max,
                   const double* pair_density, uint64_t n_frames, double* g) {
  const double pi = 3.14159265358979323846;
  const double dr = r_max / (double)nbins;
  for (int32_t h = 0; h < n_hist; ++h)
    for (int32_t k = 0; k < nbins; ++k) {
      double r0 = (double)k * dr;
      double r1 = (double)(k + 1) * dr;
      double shell = 4.0 * pi / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0);
      double per_frame = (double)counts[(size_t)h * nbins + k] / (double)n_frames;
      g[(size_t)h * nbins + k] = per_frame / (pair_density[h] * shell);
    }
}

// The same for binary64 coordinates.
void dh_oracle_pairs_r2_f64(const double* coords, const int64_t* ii, const int64_t* jj, int64_t m,
                            int32_t box_type, const double* box, double* out) {
  double zero[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  Box b = make_box(box_type, box ? box : zero);
  for (int64_t p = 0; p < m; ++p) out[p] = pair_r2(coords + 3 * ii[p], coords + 3 * jj[p], b);
}

int dh_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
