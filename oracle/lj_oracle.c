/*
 * lj_oracle.c -- plain, slow, FP64 CPU oracle for the Lennard-Jones short-range
 * force path of "Tuning of Vectorization Parameters for Molecular Dynamics
 * Simulations in AutoPas" (arXiv 2512.03565).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg (and its `--impl reference` arm) use it.  It shares no code, header,
 * table or constant generator with the CUDA library; it is written directly
 * from the paper's definitions:
 *
 *   - Sec. 2.1, Eq. (1): F_i = sum_j F_ij over all other particles.
 *   - Sec. 2.1: only pairs within the cutoff interact; Newton's third law
 *     F_ij = -F_ji.
 *   - Sec. 4.1 (Algorithm 1 names the kernel "ForceKernel"; the paper names the
 *     Lennard-Jones potential but does not print it): textbook 12-6 form
 *     U(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6], single species, truncated at
 *     r_c (not shifted).
 *   - Sec. 2.1.1: Linked Cells (cells of equal size, own + neighbour cells) and
 *     Verlet lists with a skin (cutoff + skin), rebuilt every few steps.
 *   - Sec. 2.1: velocity-Verlet integration of Newton's equations.
 *   - Sec. 6 (future work, data-driven tuning): the tuner MLP's FP64 forward,
 *     backward and Adam step.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes):
 *   R1 positions are 32-bit fixed point per axis in a cubic periodic box:
 *      x = x_fp * u with u = L / 2^32.  The minimum-image difference of two
 *      particles is the wrapping 32-bit difference read as signed.
 *   R2 a pair {i,j} interacts iff 0 < R^2 <= floor((r_c/u)^2), with R^2 the
 *      exact integer sum of squared fixed-point differences (uint64).  Pairs at
 *      zero separation are excluded.  The same integer rule (with r_c + skin)
 *      defines Verlet-list membership.
 *   R3 cells: n_c = floor(L / edge_min) per axis; cell of a coordinate is
 *      (x_fp * n_c) >> 32; linear id (cz*n_c + cy)*n_c + cx; the sort by cell
 *      is stable (ties keep ascending original index).
 *   R4 Verlet-list order: the 9 (dz,dy) rows in lexicographic order, inside a
 *      row ascending sorted index; half lists keep only j > i (sorted index).
 *   R19 Verlet cluster lists: towers, cluster order, boxes and the cluster
 *      neighbour rule, stated at orc_vcl_order below.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Fixed point and the integer cutoff threshold (readings R1, R2).           */
/* ------------------------------------------------------------------------ */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* floor((r / u)^2) with u = L / 2^32, evaluated exactly in integer arithmetic
 * from the binary expansions of r and L.  Returns UINT64_MAX on overflow. */
uint64_t orc_cut2_int(double L, double r) {
  int er, eL;
  double fr = frexp(r, &er), fL = frexp(L, &eL); /* r = fr 2^er, 0.5 <= fr < 1 */
  uint64_t mr = (uint64_t)ldexp(fr, 53), mL = (uint64_t)ldexp(fL, 53);
  /* (r/u)^2 = (mr/mL)^2 * 2^(2 er - 2 eL + 64) */
  int k = 2 * er - 2 * eL + 64;
  unsigned __int128 num = (unsigned __int128)mr * mr, den = (unsigned __int128)mL * mL;
  unsigned __int128 q = num / den, rem = num % den;
  if (k >= 0) {
    for (int i = 0; i < k; ++i) {
      rem <<= 1;
      unsigned bit = rem >= den;
      if (bit) rem -= den;
      q = (q << 1) | bit;
      if (q >> 64) return UINT64_MAX;
    }
  } else {
    q = (-k >= 128) ? 0 : (q >> (-k));
  }
  return (uint64_t)q;
}

static inline int32_t mimg(uint32_t xi, uint32_t xj) { return (int32_t)(xj - xi); }

static inline uint64_t r2int(int32_t a, int32_t b, int32_t c) {
  return (uint64_t)((int64_t)a * a) + (uint64_t)((int64_t)b * b) + (uint64_t)((int64_t)c * c);
}

uint64_t orc_r2_int(uint32_t xi, uint32_t yi, uint32_t zi, uint32_t xj, uint32_t yj, uint32_t zj) {
  return r2int(mimg(xi, xj), mimg(yi, yj), mimg(zi, zj));
}

/* Quantise a coordinate to fixed point: x_fp = floor(x / L * 2^32) mod 2^32. */
uint32_t orc_quantize(double x, double L) {
  double t = x / L;
  t = t - floor(t);
  double s = floor(ldexp(t, 32));
  if (s >= 4294967296.0) s = 0.0;
  return (uint32_t)s;
}

/* ------------------------------------------------------------------------ */
/* The pair kernel (textbook LJ 12-6, truncated) and brute-force forces.     */
/* ------------------------------------------------------------------------ */

/* Force and energy of one pair with fixed-point difference (di,dj,dk) from i to
 * j.  Adds -fac*dx to f (the force on i), returns U and W = fac * r^2. */
static inline void lj_pair(int32_t a, int32_t b, int32_t c, double u, double eps, double sig2,
                           double* f, double* U, double* W) {
  double dx = (double)a * u, dy = (double)b * u, dz = (double)c * u;
  double r2 = dx * dx + dy * dy + dz * dz;
  double s2 = sig2 / r2;
  double s6 = s2 * s2 * s2;
  double fac = 24.0 * eps * s6 * (2.0 * s6 - 1.0) / r2;
  f[0] -= fac * dx;
  f[1] -= fac * dy;
  f[2] -= fac * dz;
  *U += 4.0 * eps * s6 * (s6 - 1.0);
  *W += fac * r2;
}

/* Brute force O(N^2), minimum image, every i against every j != i (Eq. 1).
 * f: 3 arrays of n (SoA).  energy/virial count each unordered pair once.
 * Returns the number of unique in-cutoff pairs. */
int64_t orc_forces_bruteforce(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z,
                              double L, double rc, double eps, double sigma,
                              double* fx, double* fy, double* fz, double* energy, double* virial) {
  const double u = ldexp(L, -32), sig2 = sigma * sigma;
  const uint64_t Rc2 = orc_cut2_int(L, rc);
  double Utot = 0.0, Wtot = 0.0;
  int64_t npairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : Utot, Wtot, npairs)
  for (int64_t i = 0; i < n; ++i) {
    double f[3] = {0.0, 0.0, 0.0}, U = 0.0, W = 0.0;
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      int32_t a = mimg(x[i], x[j]), b = mimg(y[i], y[j]), c = mimg(z[i], z[j]);
      uint64_t R2 = r2int(a, b, c);
      if (R2 == 0 || R2 > Rc2) continue;
      lj_pair(a, b, c, u, eps, sig2, f, &U, &W);
      ++cnt;
    }
    fx[i] = f[0];
    fy[i] = f[1];
    fz[i] = f[2];
    Utot += U;
    Wtot += W;
    npairs += cnt;
  }
  if (energy) *energy = 0.5 * Utot;
  if (virial) *virial = 0.5 * Wtot;
  return npairs / 2;
}

/* Forces on a subset of particles (by index), each against all others.  Used
 * to check sampled outputs of large systems one by one. */
void orc_forces_sampled(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z,
                        double L, double rc, double eps, double sigma, int64_t nsample,
                        const int64_t* idx, double* fx, double* fy, double* fz) {
  const double u = ldexp(L, -32), sig2 = sigma * sigma;
  const uint64_t Rc2 = orc_cut2_int(L, rc);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < nsample; ++s) {
    int64_t i = idx[s];
    double f[3] = {0.0, 0.0, 0.0}, U = 0.0, W = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      int32_t a = mimg(x[i], x[j]), b = mimg(y[i], y[j]), c = mimg(z[i], z[j]);
      uint64_t R2 = r2int(a, b, c);
      if (R2 == 0 || R2 > Rc2) continue;
      lj_pair(a, b, c, u, eps, sig2, f, &U, &W);
    }
    fx[s] = f[0];
    fy[s] = f[1];
    fz[s] = f[2];
  }
}

/* All unordered pairs {i<j} with 0 < R^2 <= floor((r/u)^2), lexicographic.
 * ij may be NULL (count only); otherwise it receives 2*count int32s. */
int64_t orc_pairs_bruteforce(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z,
                             double L, double r, int32_t* ij) {
  const uint64_t R2max = orc_cut2_int(L, r);
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      uint64_t R2 = r2int(mimg(x[i], x[j]), mimg(y[i], y[j]), mimg(z[i], z[j]));
      if (R2 == 0 || R2 > R2max) continue;
      if (ij) {
        ij[2 * k] = (int32_t)i;
        ij[2 * k + 1] = (int32_t)j;
      }
      ++k;
    }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Linked cells (Sec. 2.1.1): stable counting sort by cell id (reading R3).  */
/* ------------------------------------------------------------------------ */

int orc_ncells(double L, double edge_min) {
  double q = floor(L / edge_min);
  return q < 1.0 ? 0 : (int)q;
}

static inline uint32_t cell_coord(uint32_t xf, int nc) {
  return (uint32_t)(((uint64_t)xf * (uint64_t)nc) >> 32);
}

uint32_t orc_cell_of(uint32_t xf, uint32_t yf, uint32_t zf, int nc) {
  return (cell_coord(zf, nc) * (uint32_t)nc + cell_coord(yf, nc)) * (uint32_t)nc + cell_coord(xf, nc);
}

/* perm[k] = original index of the k-th particle in cell order; cell_start has
 * nc^3 + 1 entries.  Within a cell, ascending original index. */
int orc_bin_cells(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z, int nc,
                  uint32_t* perm, uint32_t* cell_start) {
  int64_t ncell = (int64_t)nc * nc * nc;
  uint32_t* cnt = (uint32_t*)calloc((size_t)ncell + 1, sizeof(uint32_t));
  if (!cnt) return -1;
  for (int64_t i = 0; i < n; ++i) cnt[orc_cell_of(x[i], y[i], z[i], nc)]++;
  uint32_t acc = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    cell_start[c] = acc;
    acc += cnt[c];
    cnt[c] = cell_start[c];
  }
  cell_start[ncell] = acc;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t c = orc_cell_of(x[i], y[i], z[i], nc);
    perm[cnt[c]++] = (uint32_t)i;
  }
  free(cnt);
  return 0;
}

static int cmp_pair(const void* a, const void* b) {
  const int32_t* p = (const int32_t*)a;
  const int32_t* q = (const int32_t*)b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}

/* The 27 neighbour cells of (cx,cy,cz), periodic, in (dz,dy,dx)
 * lexicographic order.  Requires nc >= 3 so that the 27 cells are distinct. */
static void neighbour_cells(int nc, int cx, int cy, int cz, int64_t out[27]) {
  int k = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
        out[k++] = ((int64_t)z * nc + y) * nc + x;
      }
}

/* Pair set found by the linked-cell scan with cells of edge >= r: each
 * particle against every particle of its own and the 26 neighbour cells,
 * keeping 0 < R^2 <= floor((r/u)^2).  Output as original-index pairs i<j,
 * lexicographic (sorted).  Returns count, or -1 (nc < 3). */
int64_t orc_pairs_cells(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z,
                        double L, double r, int nc, int32_t* ij) {
  if (nc < 3) return -1;
  const uint64_t R2max = orc_cut2_int(L, r);
  int64_t ncell = (int64_t)nc * nc * nc;
  uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint32_t* cs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(ncell + 1));
  orc_bin_cells(n, x, y, z, nc, perm, cs);
  int64_t k = 0;
  for (int cz = 0; cz < nc; ++cz)
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx) {
        int64_t c = ((int64_t)cz * nc + cy) * nc + cx;
        for (uint32_t a = cs[c]; a < cs[c + 1]; ++a) {
          uint32_t i = perm[a];
          int64_t nbs[27];
          neighbour_cells(nc, cx, cy, cz, nbs);
          for (int t = 0; t < 27; ++t)
            for (uint32_t b = cs[nbs[t]]; b < cs[nbs[t] + 1]; ++b) {
              uint32_t j = perm[b];
              if (j <= i) continue;
              uint64_t R2 = r2int(mimg(x[i], x[j]), mimg(y[i], y[j]), mimg(z[i], z[j]));
              if (R2 == 0 || R2 > R2max) continue;
              if (ij) {
                ij[2 * k] = (int32_t)i;
                ij[2 * k + 1] = (int32_t)j;
              }
              ++k;
            }
        }
      }
  if (ij) qsort(ij, (size_t)k, 2 * sizeof(int32_t), cmp_pair);
  free(perm);
  free(cs);
  return k;
}

/* Verlet lists (Sec. 2.1.1) in sorted-index space (reading R4).  Cells of edge
 * >= r_l = rc + skin.  nbr is row-major [n][cap] of sorted j indices, nnbr[n]
 * the list lengths.  Returns 0, or 1 if some list exceeded cap (lengths are
 * still complete; entries beyond cap are dropped), or -1 on bad arguments. */
int orc_verlet(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z, double L,
               double rl, int nc, int half, int cap, uint32_t* perm, uint32_t* cell_start,
               int32_t* nbr, int32_t* nnbr) {
  if (nc < 3) return -1;
  const uint64_t R2max = orc_cut2_int(L, rl);
  orc_bin_cells(n, x, y, z, nc, perm, cell_start);
  int over = 0;
  for (int cz = 0; cz < nc; ++cz)
    for (int cy = 0; cy < nc; ++cy)
      for (int cx = 0; cx < nc; ++cx) {
        int64_t c = ((int64_t)cz * nc + cy) * nc + cx;
        for (uint32_t a = cell_start[c]; a < cell_start[c + 1]; ++a) {
          uint32_t i = perm[a];
          int cnt = 0;
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
              /* one row: the three cells (cx-1..cx+1) in ascending cell id */
              int ids[3];
              for (int t = 0; t < 3; ++t) ids[t] = (cx + t - 1 + nc) % nc;
              /* sort the three x-cells ascending */
              for (int p = 0; p < 3; ++p)
                for (int q = p + 1; q < 3; ++q)
                  if (ids[q] < ids[p]) {
                    int tmp = ids[p];
                    ids[p] = ids[q];
                    ids[q] = tmp;
                  }
              int ncy = (cy + dy + nc) % nc, ncz = (cz + dz + nc) % nc;
              for (int t = 0; t < 3; ++t) {
                int64_t nb = ((int64_t)ncz * nc + ncy) * nc + ids[t];
                for (uint32_t b = cell_start[nb]; b < cell_start[nb + 1]; ++b) {
                  if (b == a) continue;
                  if (half && b <= a) continue;
                  uint32_t j = perm[b];
                  uint64_t R2 = r2int(mimg(x[i], x[j]), mimg(y[i], y[j]), mimg(z[i], z[j]));
                  if (R2 == 0 || R2 > R2max) continue;
                  if (cnt < cap) nbr[(int64_t)a * cap + cnt] = (int32_t)b;
                  ++cnt;
                }
              }
            }
          nnbr[a] = cnt;
          if (cnt > cap) over = 1;
        }
      }
  return over;
}

/* ------------------------------------------------------------------------ */
/* Verlet cluster lists (Sec. 2.1.1: clusters of a fixed number of nearby    */
/* particles, with neighbour lists of whole clusters rebuilt every few steps; */
/* Sec. 5.1: cluster sizes 4, 6 and 8).  Reading R19:                        */
/*   - towers: n_t x n_t columns over (x, y), n_t the largest k >= 1 with    */
/*     k^3 M <= n (so a tower cell holds about M particles and a cluster is  */
/*     about as tall as it is wide); column of a particle                    */
/*     (cell_coord(x, n_t), cell_coord(y, n_t)), column id cx n_t + cy;      */
/*   - storage order: by column id, then z, then original index;             */
/*   - clusters: consecutive runs of M particles of one column, the last run */
/*     of a column shorter when its count is not a multiple of M;            */
/*   - a cluster's box is the min/max of its particles' fixed-point          */
/*     coordinates per axis (a column never wraps in x or y, and z is sorted */
/*     ascending inside it, so no box wraps);                                */
/*   - clusters I and J are neighbours iff D^2 <= floor((r_l/u)^2), where    */
/*     D^2 = sum over axes of d_a^2 and d_a is the periodic distance of the  */
/*     two boxes' intervals on the 2^32 circle (0 when they intersect);      */
/*     full lists hold every such J (I itself included), half lists those    */
/*     with J >= I.  No pair within r_l is missed: |mimg_a(x_i - x_j)| >= d_a */
/*     for every i in I and j in J.                                          */
/* ------------------------------------------------------------------------ */

int orc_vcl_ntower(int64_t n, int M) {
  if (M < 1 || n < 1) return 1;
  int64_t k = 1;
  while ((k + 1) * (k + 1) * (k + 1) * (int64_t)M <= n) ++k;
  return (int)k;
}

static const uint32_t *g_sx, *g_sy, *g_sz;
static int g_nt;
static int cmp_tower_order(const void* a, const void* b) {
  const uint32_t i = *(const uint32_t*)a, j = *(const uint32_t*)b;
  const uint64_t ci = (uint64_t)cell_coord(g_sx[i], g_nt) * (uint64_t)g_nt + cell_coord(g_sy[i], g_nt);
  const uint64_t cj = (uint64_t)cell_coord(g_sx[j], g_nt) * (uint64_t)g_nt + cell_coord(g_sy[j], g_nt);
  if (ci != cj) return ci < cj ? -1 : 1;
  if (g_sz[i] != g_sz[j]) return g_sz[i] < g_sz[j] ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

/* perm[k] = original index of the k-th particle in cluster order; cl_start
 * (capacity n + 1) receives the cluster boundaries.  Returns the number of
 * clusters, or -1 on bad arguments.  Not thread-safe (qsort comparator state). */
int64_t orc_vcl_order(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z, int M,
                      uint32_t* perm, uint32_t* cl_start) {
  if (n < 1 || M < 1) return -1;
  const int nt = orc_vcl_ntower(n, M);
  for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
  g_sx = x;
  g_sy = y;
  g_sz = z;
  g_nt = nt;
  qsort(perm, (size_t)n, sizeof(uint32_t), cmp_tower_order);
  int64_t ncl = 0, k = 0;
  while (k < n) {
    /* one column: [k, e) */
    const uint32_t p = perm[k];
    const uint32_t cx = cell_coord(x[p], nt), cy = cell_coord(y[p], nt);
    int64_t e = k;
    while (e < n && cell_coord(x[perm[e]], nt) == cx && cell_coord(y[perm[e]], nt) == cy) ++e;
    for (int64_t b = k; b < e; b += M) cl_start[ncl++] = (uint32_t)b;
    k = e;
  }
  cl_start[ncl] = (uint32_t)n;
  return ncl;
}


/* Cluster-pair lists by brute force over all cluster pairs and all their
 * member pairs (readings R19 and R21).  perm / cl_start as from
 * orc_vcl_order; x, y, z in original order.  I lists J iff some member pair
 * (the a-th particle of I, the b-th of J, two different particles) lies
 * within r_l: 0 < R^2 <= floor((r_l/u)^2).  Half lists (half = 1) keep J >= I
 * and, for J = I, the pairs with b > a.  masks (may be NULL) receives per
 * listed pair the bits a * M + b of those member pairs (M the cluster size,
 * at most 8, so 64 bits suffice; every cluster holds at most M).  nbr is row-major
 * [ncl][cap] of cluster indices in ascending order, nn[ncl] the complete list
 * lengths (entries beyond cap are dropped).  Returns 0, 1 if a list exceeded
 * cap, -1 on bad arguments. */
int orc_vcl_lists(int64_t ncl, const uint32_t* perm, const uint32_t* cl_start, const uint32_t* x,
                  const uint32_t* y, const uint32_t* z, double L, double rl, int half, int M, int cap,
                  int32_t* nbr, int32_t* nn, uint64_t* masks) {
  if (ncl < 0 || M < 1 || M > 8) return -1;
  for (int64_t c = 0; c < ncl; ++c)
    if (cl_start[c + 1] - cl_start[c] > (uint32_t)M) return -1;
  const uint64_t R2max = orc_cut2_int(L, rl);
  int over = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : over)
  for (int64_t I = 0; I < ncl; ++I) {
    int cnt = 0;
    for (int64_t J = half ? I : 0; J < ncl; ++J) {
      uint64_t mask = 0;
      for (uint32_t a = 0; a < cl_start[I + 1] - cl_start[I]; ++a) {
        const uint32_t p = perm[cl_start[I] + a];
        for (uint32_t b = 0; b < cl_start[J + 1] - cl_start[J]; ++b) {
          if (J == I && (half ? b <= a : b == a)) continue;
          const uint32_t q = perm[cl_start[J] + b];
          const uint64_t R2 = r2int(mimg(x[p], x[q]), mimg(y[p], y[q]), mimg(z[p], z[q]));
          if (R2 != 0 && R2 <= R2max) mask |= 1ull << (a * (uint32_t)M + b);
        }
      }
      if (!mask) continue;
      if (cnt < cap) {
        nbr[I * cap + cnt] = (int32_t)J;
        if (masks) masks[I * cap + cnt] = mask;
      }
      ++cnt;
    }
    nn[I] = cnt;
    if (cnt > cap) over = 1;
  }
  return over;
}

/* Linked-cell forces (FP64), the CPU baseline for large systems: identical
 * result to the brute force up to summation order.  Each particle visits its
 * 27 neighbour cells (no Newton-3 halving; every pair is evaluated twice). */
int64_t orc_forces_cells(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z,
                         double L, double rc, double eps, double sigma, double* fx, double* fy,
                         double* fz, double* energy, double* virial) {
  int nc = orc_ncells(L, rc);
  if (nc < 3) return -1;
  const double u = ldexp(L, -32), sig2 = sigma * sigma;
  const uint64_t Rc2 = orc_cut2_int(L, rc);
  int64_t ncell = (int64_t)nc * nc * nc;
  uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint32_t* cs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(ncell + 1));
  orc_bin_cells(n, x, y, z, nc, perm, cs);
  double Utot = 0.0, Wtot = 0.0;
  int64_t npairs = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : Utot, Wtot, npairs)
  for (int64_t c = 0; c < ncell; ++c) {
    int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
    for (uint32_t a = cs[c]; a < cs[c + 1]; ++a) {
      uint32_t i = perm[a];
      double f[3] = {0.0, 0.0, 0.0}, U = 0.0, W = 0.0;
      int64_t cnt = 0;
      int64_t nbs[27];
      neighbour_cells(nc, cx, cy, cz, nbs);
      for (int t = 0; t < 27; ++t)
        for (uint32_t b = cs[nbs[t]]; b < cs[nbs[t] + 1]; ++b) {
          uint32_t j = perm[b];
          if (j == i) continue;
          int32_t p = mimg(x[i], x[j]), q = mimg(y[i], y[j]), r = mimg(z[i], z[j]);
          uint64_t R2 = r2int(p, q, r);
          if (R2 == 0 || R2 > Rc2) continue;
          lj_pair(p, q, r, u, eps, sig2, f, &U, &W);
          ++cnt;
        }
      fx[i] = f[0];
      fy[i] = f[1];
      fz[i] = f[2];
      Utot += U;
      Wtot += W;
      npairs += cnt;
    }
  }
  free(perm);
  free(cs);
  if (energy) *energy = 0.5 * Utot;
  if (virial) *virial = 0.5 * Wtot;
  return npairs / 2;
}

/* ------------------------------------------------------------------------ */
/* Velocity Verlet (Sec. 2.1).                                               */
/* ------------------------------------------------------------------------ */

/* nsteps of: v += (dt/2m) F; x_fp += rne(v * (dt 2^32/L)) (mod 2^32, the
 * periodic wrap); F = F(x); v += (dt/2m) F.  Each kick is one correctly
 * rounded fma(dt/2m, F, v).  The displacement in fixed-point units is the
 * exact product v * dtu rounded once to the nearest integer (ties to even):
 * fma(v, dtu, 1.5 2^52) - 1.5 2^52, valid for |v dtu| < 2^51.  f must hold
 * the forces at the initial positions on entry and holds those at the final
 * positions on exit.  use_cells selects the linked-cell force routine (else
 * brute force). */
int orc_vv_run(int64_t n, uint32_t* x, uint32_t* y, uint32_t* z, double* vx, double* vy,
               double* vz, double* fx, double* fy, double* fz, double mass, double dt, int nsteps,
               double L, double rc, double eps, double sigma, int use_cells, double* energy,
               double* virial) {
  const double hdtm = 0.5 * dt / mass;
  const double dtu = dt * ldexp(1.0, 32) / L;
  uint32_t* xyz[3] = {x, y, z};
  double* v[3] = {vx, vy, vz};
  double* f[3] = {fx, fy, fz};
  for (int s = 0; s < nsteps; ++s) {
    for (int a = 0; a < 3; ++a)
      for (int64_t i = 0; i < n; ++i) {
        v[a][i] = fma(hdtm, f[a][i], v[a][i]);
        double d = fma(v[a][i], dtu, 6755399441055744.0) - 6755399441055744.0;
        xyz[a][i] = xyz[a][i] + (uint32_t)(uint64_t)(int64_t)d;
      }
    int64_t r;
    if (use_cells)
      r = orc_forces_cells(n, x, y, z, L, rc, eps, sigma, fx, fy, fz, energy, virial);
    else
      r = orc_forces_bruteforce(n, x, y, z, L, rc, eps, sigma, fx, fy, fz, energy, virial);
    if (r < 0) return -1;
    for (int a = 0; a < 3; ++a)
      for (int64_t i = 0; i < n; ++i) v[a][i] = fma(hdtm, f[a][i], v[a][i]);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tuner features (no counterpart in the paper; Sec. 6 asks for data-driven  */
/* tuning).  16 features from the linked-cell occupancy (cells of edge rc).  */
/* ------------------------------------------------------------------------ */

/* out[16]:
 *  0 log(rho)            1 log(N)              2 mean cell occupancy
 *  3 std occupancy       4 fraction of empty cells
 *  5..12 occupancy histogram, bins {0},{1-2},{3-4},{5-8},{9-16},{17-32},
 *        {33-64},{>64}, as fractions of cells
 *  13 homogeneity: std/mean of counts over the 4x4x4 coarse blocks given by
 *     the top two bits of each fixed-point coordinate
 *  14 rc / cell edge     15 expected Verlet-list length:
 *     (sum_c occ_c^2 / N) * (4/3 pi rl^3) / cell volume                    */
int orc_features(int64_t n, const uint32_t* x, const uint32_t* y, const uint32_t* z, double L,
                 double rc, double skin, double* out) {
  int nc = orc_ncells(L, rc);
  if (nc < 1 || n < 1) return -1;
  int64_t ncell = (int64_t)nc * nc * nc;
  uint32_t* occ = (uint32_t*)calloc((size_t)ncell, sizeof(uint32_t));
  int64_t blocks[64];
  memset(blocks, 0, sizeof(blocks));
  for (int64_t i = 0; i < n; ++i) {
    occ[orc_cell_of(x[i], y[i], z[i], nc)]++;
    blocks[((z[i] >> 30) * 4 + (y[i] >> 30)) * 4 + (x[i] >> 30)]++;
  }
  double s1 = 0.0, s2 = 0.0;
  int64_t hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t c = 0; c < ncell; ++c) {
    uint32_t o = occ[c];
    s1 += (double)o;
    s2 += (double)o * (double)o;
    int b = o == 0 ? 0 : o <= 2 ? 1 : o <= 4 ? 2 : o <= 8 ? 3 : o <= 16 ? 4 : o <= 32 ? 5 : o <= 64 ? 6 : 7;
    hist[b]++;
  }
  free(occ);
  double mean = s1 / (double)ncell;
  double var = s2 / (double)ncell - mean * mean;
  double bm = (double)n / 64.0, bv = 0.0;
  for (int b = 0; b < 64; ++b) bv += ((double)blocks[b] - bm) * ((double)blocks[b] - bm);
  bv /= 64.0;
  const double pi = 3.14159265358979323846;
  double edge = L / (double)nc;
  double rl = rc + skin;
  out[0] = log((double)n / (L * L * L));
  out[1] = log((double)n);
  out[2] = mean;
  out[3] = sqrt(var > 0.0 ? var : 0.0);
  out[4] = (double)hist[0] / (double)ncell;
  for (int b = 0; b < 8; ++b) out[5 + b] = (double)hist[b] / (double)ncell;
  out[13] = sqrt(bv) / bm;
  out[14] = rc / edge;
  out[15] = (s2 / (double)n) * (4.0 / 3.0 * pi * rl * rl * rl) / (edge * edge * edge);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tuner MLP, FP64: in(16) -> tanh(64) -> tanh(64) -> linear(C).             */
/* Parameter layout: W1[64][16] b1[64] W2[64][64] b2[64] W3[C][64] b3[C].    */
/* Loss: sum_rc m_rc (yhat_rc - y_rc)^2 / sum_rc m_rc (masked MSE).          */
/* ------------------------------------------------------------------------ */

#define MLP_IN 16
#define MLP_H 64

int64_t orc_mlp_nparams(int C) {
  return (int64_t)MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + (int64_t)C * MLP_H + C;
}

/* Forward for M rows: X[M][16] -> Y[M][C]. */
void orc_mlp_forward(const double* p, int C, int64_t M, const double* X, double* Y) {
  const double *W1 = p, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
  const double *W3 = b2 + MLP_H, *b3 = W3 + (int64_t)C * MLP_H;
  for (int64_t m = 0; m < M; ++m) {
    double h1[MLP_H], h2[MLP_H];
    for (int o = 0; o < MLP_H; ++o) {
      double s = b1[o];
      for (int i = 0; i < MLP_IN; ++i) s += W1[o * MLP_IN + i] * X[m * MLP_IN + i];
      h1[o] = tanh(s);
    }
    for (int o = 0; o < MLP_H; ++o) {
      double s = b2[o];
      for (int i = 0; i < MLP_H; ++i) s += W2[o * MLP_H + i] * h1[i];
      h2[o] = tanh(s);
    }
    for (int o = 0; o < C; ++o) {
      double s = b3[o];
      for (int i = 0; i < MLP_H; ++i) s += W3[o * MLP_H + i] * h2[i];
      Y[m * C + o] = s;
    }
  }
}

/* Loss and its gradient with respect to every parameter (backpropagation). */
double orc_mlp_loss_grad(const double* p, int C, int64_t M, const double* X, const double* T,
                         const double* mask, double* grad) {
  const double *W1 = p, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
  const double *W3 = b2 + MLP_H;
  const double* b3 = W3 + (int64_t)C * MLP_H;
  int64_t P = orc_mlp_nparams(C);
  double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
  double *gW3 = gb2 + MLP_H, *gb3 = gW3 + (int64_t)C * MLP_H;
  memset(grad, 0, sizeof(double) * (size_t)P);
  double msum = 0.0;
  for (int64_t k = 0; k < M * C; ++k) msum += mask[k];
  if (msum <= 0.0) return 0.0;
  double loss = 0.0;
  double* y = (double*)malloc(sizeof(double) * (size_t)C);
  double* dy = (double*)malloc(sizeof(double) * (size_t)C);
  for (int64_t m = 0; m < M; ++m) {
    const double* x = X + m * MLP_IN;
    double h1[MLP_H], h2[MLP_H], d1[MLP_H], d2[MLP_H];
    for (int o = 0; o < MLP_H; ++o) {
      double s = b1[o];
      for (int i = 0; i < MLP_IN; ++i) s += W1[o * MLP_IN + i] * x[i];
      h1[o] = tanh(s);
    }
    for (int o = 0; o < MLP_H; ++o) {
      double s = b2[o];
      for (int i = 0; i < MLP_H; ++i) s += W2[o * MLP_H + i] * h1[i];
      h2[o] = tanh(s);
    }
    for (int o = 0; o < C; ++o) {
      double s = b3[o];
      for (int i = 0; i < MLP_H; ++i) s += W3[o * MLP_H + i] * h2[i];
      y[o] = s;
      double e = s - T[m * C + o];
      loss += mask[m * C + o] * e * e;
      dy[o] = 2.0 * mask[m * C + o] * e / msum;
    }
    for (int i = 0; i < MLP_H; ++i) d2[i] = 0.0;
    for (int o = 0; o < C; ++o) {
      gb3[o] += dy[o];
      for (int i = 0; i < MLP_H; ++i) {
        gW3[o * MLP_H + i] += dy[o] * h2[i];
        d2[i] += dy[o] * W3[o * MLP_H + i];
      }
    }
    for (int i = 0; i < MLP_H; ++i) d2[i] *= (1.0 - h2[i] * h2[i]);
    for (int i = 0; i < MLP_H; ++i) d1[i] = 0.0;
    for (int o = 0; o < MLP_H; ++o) {
      gb2[o] += d2[o];
      for (int i = 0; i < MLP_H; ++i) {
        gW2[o * MLP_H + i] += d2[o] * h1[i];
        d1[i] += d2[o] * W2[o * MLP_H + i];
      }
    }
    for (int i = 0; i < MLP_H; ++i) d1[i] *= (1.0 - h1[i] * h1[i]);
    for (int o = 0; o < MLP_H; ++o) {
      gb1[o] += d1[o];
      for (int i = 0; i < MLP_IN; ++i) gW1[o * MLP_IN + i] += d1[o] * x[i];
    }
  }
  free(y);
  free(dy);
  return loss / msum;
}

/* One Adam step (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).  t counts from 1. */
void orc_adam_step(int64_t P, double* p, const double* g, double* m, double* v, double lr,
                   double beta1, double beta2, double eps, int t) {
  double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  for (int64_t k = 0; k < P; ++k) {
    m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
    v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
    p[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
  }
}

/* Training targets of the learned tuner (data-driven tuning, Sec. 6): per row
 * m of timings T[M][C] (a configuration not timed is NaN, or not positive),
 * the relative log time Y = log(T / t_best) with t_best the row's smallest
 * valid time, and mask = 1 where valid (Y = 0, mask = 0 elsewhere). */
void orc_tuner_targets(int64_t M, int C, const double* T, double* Y, double* mask) {
  for (int64_t m = 0; m < M; ++m) {
    double best = INFINITY;
    for (int c = 0; c < C; ++c) {
      const double t = T[m * C + c];
      if (isfinite(t) && t > 0.0 && t < best) best = t;
    }
    for (int c = 0; c < C; ++c) {
      const double t = T[m * C + c];
      const int ok = isfinite(t) && t > 0.0;
      Y[m * C + c] = ok ? log(t / best) : 0.0;
      mask[m * C + c] = ok ? 1.0 : 0.0;
    }
  }
}

/* Feature standardisation of the tuner: mean and (population) standard
 * deviation of each of the F columns of X[M][F] over the rows, a deviation
 * below 1e-12 replaced by 1, and Xs = (X - mean) / std. */
void orc_standardize(int64_t M, int F, const double* X, double* Xs, double* mean, double* sd) {
  for (int f = 0; f < F; ++f) {
    double s = 0.0;
    for (int64_t m = 0; m < M; ++m) s += X[m * F + f];
    const double mu = s / (double)M;
    double q = 0.0;
    for (int64_t m = 0; m < M; ++m) q += (X[m * F + f] - mu) * (X[m * F + f] - mu);
    double sig = sqrt(q / (double)M);
    if (sig < 1e-12) sig = 1.0;
    mean[f] = mu;
    sd[f] = sig;
    for (int64_t m = 0; m < M; ++m) Xs[m * F + f] = (X[m * F + f] - mu) / sig;
  }
}
