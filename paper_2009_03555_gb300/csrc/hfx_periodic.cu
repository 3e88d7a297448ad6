// hfx_periodic.cu -- periodic systems as an extended atom set (host code).
//
// Sec. 2, Eq. H-HFX: for a periodic system the exchange matrix is
//   K^G_{mu lambda} = sum_{N,H} sum_{nu sigma} P^{H-N}_{nu sigma} (mu^0 nu^N | lambda^G sigma^H),
// mu in the home cell and nu, lambda, sigma in the cells N, G, H of the
// auxiliary supercell.  Here the supercell is an extended atom set: the home
// atoms followed by the images (translates of home atoms by lattice vectors)
// that lie within r_ext of some home atom.  Each image carries its home atom's
// shells.  The sum above is then the row of mu^0 (column lambda^G) of the
// molecular exchange of the extended set; a periodic basis
// (hfx_create_basis_periodic, hfx_core.cu) evaluates only the quartets with a
// home-cell shell, which are the ones that reach those rows.  These functions
// produce the image table, the extended set, the distance pattern and lay the
// real-space density P^{H-N} onto the extended pattern.
//
// Real-space density at the Gamma point (Eq. dm with one k-point): the
// caller's pattern over the extended atoms decides where P^{H-N} is nonzero
// (normally the atom pairs within a distance cutoff, hfx_distance_pattern).
// Every block (X, Y) of that pattern receives the home-cell density block of
// the home atoms of X and Y.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hfx.h"

void hfx_set_last_error(const std::string& m);

namespace {

long long periodic_fail(const std::string& m) {
  hfx_set_last_error(m);
  return -1;
}

hfx_status status_fail(hfx_status s, const std::string& m) {
  hfx_set_last_error(m);
  return s;
}

int n_cart(int l) { return (l + 1) * (l + 2) / 2; }

}  // namespace

extern "C" {

long long hfx_periodic_images(const double* atom_xyz, int n_atoms, const double* lattice, double r_ext,
                              long long max_images, int* image_atom, int* image_shift) {
  if (!atom_xyz || !lattice || n_atoms <= 0) return periodic_fail("hfx_periodic_images: NULL argument or no atoms");
  if (!(r_ext >= 0.0) || !std::isfinite(r_ext)) return periodic_fail("hfx_periodic_images: r_ext must be >= 0");
  if (max_images > 0 && (!image_atom || !image_shift))
    return periodic_fail("hfx_periodic_images: NULL output arrays");
  const double* a = lattice;
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return periodic_fail("hfx_periodic_images: singular lattice");
  // |n_i| = |L . b_i| <= |L| |b_i| with b_i = (a_j x a_k) / det; a kept image
  // has |L| <= r_ext + (largest distance between home atoms)
  double diam2 = 0.0;
  for (int p = 0; p < n_atoms; ++p)
    for (int q = p + 1; q < n_atoms; ++q) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) d2 += (atom_xyz[3 * p + k] - atom_xyz[3 * q + k]) * (atom_xyz[3 * p + k] - atom_xyz[3 * q + k]);
      diam2 = std::max(diam2, d2);
    }
  const double reach = r_ext + std::sqrt(diam2);
  int m[3];
  long long n_shift = 1;
  for (int i = 0; i < 3; ++i) {
    const double* aj = a + 3 * ((i + 1) % 3);
    const double* ak = a + 3 * ((i + 2) % 3);
    const double c0 = aj[1] * ak[2] - aj[2] * ak[1], c1 = aj[2] * ak[0] - aj[0] * ak[2],
                 c2 = aj[0] * ak[1] - aj[1] * ak[0];
    const double bnorm = std::sqrt(c0 * c0 + c1 * c1 + c2 * c2) / std::fabs(det);
    const double mi = std::floor(reach * bnorm) + 1.0;
    if (mi > 1000.0) return periodic_fail("hfx_periodic_images: r_ext too large for this lattice");
    m[i] = (int)mi;
    n_shift *= 2LL * m[i] + 1;
  }
  if (n_shift * n_atoms * (long long)n_atoms > 4000000000LL)
    return periodic_fail("hfx_periodic_images: search too large (r_ext or atom count)");
  // shift-major order: (n1, n2, n3) lexicographic, then atoms ascending
  long long count = 0;
  for (int n1 = -m[0]; n1 <= m[0]; ++n1)
    for (int n2 = -m[1]; n2 <= m[1]; ++n2)
      for (int n3 = -m[2]; n3 <= m[2]; ++n3) {
        if (n1 == 0 && n2 == 0 && n3 == 0) continue;
        for (int p = 0; p < n_atoms; ++p) {
          double x[3];
          for (int k = 0; k < 3; ++k)
            x[k] = atom_xyz[3 * p + k] + n1 * lattice[k] + n2 * lattice[3 + k] + n3 * lattice[6 + k];
          bool near = false;
          for (int q = 0; q < n_atoms && !near; ++q) {
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) d2 += (x[k] - atom_xyz[3 * q + k]) * (x[k] - atom_xyz[3 * q + k]);
            near = std::sqrt(d2) <= r_ext;
          }
          if (!near) continue;
          if (count < max_images) {
            image_atom[count] = p;
            image_shift[3 * count + 0] = n1;
            image_shift[3 * count + 1] = n2;
            image_shift[3 * count + 2] = n3;
          }
          ++count;
        }
      }
  return count;
}

long long hfx_periodic_extend(const double* atom_xyz, int n_atoms, const double* lattice, double r_ext,
                              long long max_atoms, int* ext_home, int* ext_shift, double* ext_xyz) {
  if (max_atoms > 0 && (!ext_home || !ext_shift || !ext_xyz))
    return periodic_fail("hfx_periodic_extend: NULL output arrays");
  const long long n_img = hfx_periodic_images(atom_xyz, n_atoms, lattice, r_ext, 0, nullptr, nullptr);
  if (n_img < 0) return -1;  // message set by hfx_periodic_images
  const long long n_ext = n_atoms + n_img;
  if (max_atoms <= 0) return n_ext;
  std::vector<int> atom((size_t)std::max<long long>(n_img, 1)), shift(3 * (size_t)std::max<long long>(n_img, 1));
  if (n_img > 0 && hfx_periodic_images(atom_xyz, n_atoms, lattice, r_ext, n_img, atom.data(), shift.data()) != n_img)
    return periodic_fail("hfx_periodic_extend: image table changed between calls");
  for (long long X = 0; X < n_ext && X < max_atoms; ++X) {
    const bool home = X < n_atoms;
    const int h = home ? (int)X : atom[(size_t)(X - n_atoms)];
    const int* n = home ? nullptr : &shift[3 * (size_t)(X - n_atoms)];
    ext_home[X] = h;
    for (int k = 0; k < 3; ++k) {
      ext_shift[3 * X + k] = home ? 0 : n[k];
      // R_X = R_h + n1 a1 + n2 a2 + n3 a3 (lattice vectors as rows)
      ext_xyz[3 * X + k] = atom_xyz[3 * h + k] +
                           (home ? 0.0 : n[0] * lattice[k] + n[1] * lattice[3 + k] + n[2] * lattice[6 + k]);
    }
  }
  return n_ext;
}

long long hfx_distance_pattern(const double* atom_xyz, int n_atoms, double r_cut, int* row_ptr, int* col,
                               long long max_nnz) {
  if (!atom_xyz || n_atoms <= 0 || !(r_cut >= 0.0) || !std::isfinite(r_cut))
    return periodic_fail("hfx_distance_pattern: NULL coordinates, no atoms or a bad cutoff");
  const double r2 = r_cut * r_cut;
  long long nnz = 0;
  if (row_ptr) row_ptr[0] = 0;
  for (int X = 0; X < n_atoms; ++X) {
    for (int Y = 0; Y < n_atoms; ++Y) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) d2 += (atom_xyz[3 * X + k] - atom_xyz[3 * Y + k]) * (atom_xyz[3 * X + k] - atom_xyz[3 * Y + k]);
      if (d2 <= r2 || X == Y) {
        if (col && nnz < max_nnz) col[nnz] = Y;
        ++nnz;
      }
    }
    if (nnz > (1LL << 31) - 1) return periodic_fail("hfx_distance_pattern: more than 2^31 - 1 pairs");
    if (row_ptr) row_ptr[X + 1] = (int)nnz;
  }
  return nnz;
}

hfx_status hfx_periodic_pack_lattice_host(const hfx_shell_desc* shells, int n_shells, int n_home_atoms,
                                          const int* ext_home, const int* ext_shift, const hfx_pattern* ext_pattern,
                                          int n_L, const int* L_shift, const double* P_L, double* val) {
  if (!shells || n_shells <= 0 || n_home_atoms <= 0 || !ext_home || !ext_shift || !ext_pattern ||
      !ext_pattern->row_ptr || !ext_pattern->col || ext_pattern->n_atoms <= 0 || n_L < 0 ||
      (n_L > 0 && (!L_shift || !P_L)) || !val)
    return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_lattice_host: NULL or empty argument");
  std::vector<long long> nf((size_t)n_home_atoms, 0), f0((size_t)n_home_atoms + 1, 0);
  for (int s = 0; s < n_shells; ++s) {
    const int at = shells[s].atom, l = shells[s].l;
    if (at < 0 || at >= n_home_atoms || l < 0 || l > 2 || (s > 0 && at < shells[s - 1].atom))
      return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_lattice_host: shells not grouped by home atom");
    nf[(size_t)at] += n_cart(l);
  }
  for (int at = 0; at < n_home_atoms; ++at) f0[(size_t)at + 1] = f0[(size_t)at] + nf[(size_t)at];
  const long long nbf = f0[(size_t)n_home_atoms];
  const int n_ext = ext_pattern->n_atoms;
  for (int X = 0; X < n_ext; ++X)
    if (ext_home[X] < 0 || ext_home[X] >= n_home_atoms)
      return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_lattice_host: ext_home out of range");
  long long v = 0;
  for (int X = 0; X < n_ext; ++X) {
    if (ext_pattern->row_ptr[X] > ext_pattern->row_ptr[X + 1])
      return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_lattice_host: row_ptr not ascending");
    const int hx = ext_home[X];
    for (int k = ext_pattern->row_ptr[X]; k < ext_pattern->row_ptr[X + 1]; ++k) {
      const int Y = ext_pattern->col[k];
      if (Y < 0 || Y >= n_ext)
        return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_lattice_host: column out of range");
      const int hy = ext_home[Y];
      // P^{H-N}: the lattice vector from the cell of X (N) to the cell of Y (H)
      int L = -1;
      for (int l = 0; l < n_L && L < 0; ++l)
        if (L_shift[3 * l] == ext_shift[3 * Y] - ext_shift[3 * X] &&
            L_shift[3 * l + 1] == ext_shift[3 * Y + 1] - ext_shift[3 * X + 1] &&
            L_shift[3 * l + 2] == ext_shift[3 * Y + 2] - ext_shift[3 * X + 2])
          L = l;
      const double* PL = L >= 0 ? P_L + (size_t)L * (size_t)nbf * (size_t)nbf : nullptr;
      for (long long i = 0; i < nf[(size_t)hx]; ++i)
        for (long long j = 0; j < nf[(size_t)hy]; ++j)
          val[v++] = PL ? PL[(f0[(size_t)hx] + i) * nbf + f0[(size_t)hy] + j] : 0.0;
    }
  }
  return HFX_OK;
}

hfx_status hfx_periodic_pack_host(const hfx_shell_desc* shells, int n_shells, int n_home_atoms, const int* ext_home,
                                  const hfx_pattern* ext_pattern, const double* P_home, double* val) {
  if (!shells || n_shells <= 0 || n_home_atoms <= 0 || !ext_home || !ext_pattern || !ext_pattern->row_ptr ||
      !ext_pattern->col || ext_pattern->n_atoms <= 0 || !P_home || !val)
    return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_host: NULL or empty argument");
  // home atom -> first function and function count (shells grouped by atom)
  std::vector<long long> nf((size_t)n_home_atoms, 0), f0((size_t)n_home_atoms + 1, 0);
  for (int s = 0; s < n_shells; ++s) {
    const int at = shells[s].atom, l = shells[s].l;
    if (at < 0 || at >= n_home_atoms || l < 0 || l > 2 || (s > 0 && at < shells[s - 1].atom))
      return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_host: shells not grouped by home atom");
    nf[(size_t)at] += n_cart(l);
  }
  for (int at = 0; at < n_home_atoms; ++at) f0[(size_t)at + 1] = f0[(size_t)at] + nf[(size_t)at];
  const long long nbf = f0[(size_t)n_home_atoms];
  const int n_ext = ext_pattern->n_atoms;
  for (int X = 0; X < n_ext; ++X)
    if (ext_home[X] < 0 || ext_home[X] >= n_home_atoms)
      return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_host: ext_home out of range");
  long long v = 0;
  for (int X = 0; X < n_ext; ++X) {
    if (ext_pattern->row_ptr[X] > ext_pattern->row_ptr[X + 1])
      return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_host: row_ptr not ascending");
    const int hx = ext_home[X];
    for (int k = ext_pattern->row_ptr[X]; k < ext_pattern->row_ptr[X + 1]; ++k) {
      const int Y = ext_pattern->col[k];
      if (Y < 0 || Y >= n_ext) return status_fail(HFX_ERR_INVALID_ARG, "hfx_periodic_pack_host: column out of range");
      const int hy = ext_home[Y];
      for (long long i = 0; i < nf[(size_t)hx]; ++i)
        for (long long j = 0; j < nf[(size_t)hy]; ++j) val[v++] = P_home[(f0[(size_t)hx] + i) * nbf + f0[(size_t)hy] + j];
    }
  }
  return HFX_OK;
}

}  // extern "C"
