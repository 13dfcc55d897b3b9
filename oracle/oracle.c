/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the batched pair-potential
 * MD / FIRE / adjoint path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file; only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py use it (through oracle/oracle.py).
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every function follows a written definition, cited at the function:
 *   - TorchSim (arXiv 2508.06628) Sec. 3: SimState concatenation of atom-wise
 *     arrays and stacking of system-wise arrays, indexed by a system index;
 *     Sec. 2: energies, forces and stress as the model output; differentiable
 *     trajectories with an RDF observable; Sec. 4: Langevin MD.
 *   - The paper names Lennard-Jones, Morse and soft-sphere potentials without
 *     formulas; the textbook forms are used (soft sphere as in JAX MD, the
 *     paper's ref. [12]).
 *   - Velocity Verlet (Swope et al. 1982), BAOAB Langevin (Leimkuhler and
 *     Matthews 2013), FIRE (Bitzek et al., PRL 97, 170201, 2006),
 *     Philox4x32-10 (Salmon et al., SC'11), Box-Muller (1958).
 * Precision: FP64 everywhere.  Units: Angstrom, eV, amu; time unit
 * t0 = sqrt(amu*A^2/eV) = 10.1805 fs.  Cells are 3x3 row-major with rows =
 * lattice vectors, so a fractional row vector s maps to x = s h.
 *
 * Parity status of each function is stated in its comment ("pinned by" lists
 * the independent checks in tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Potentials.  kind 0 = Lennard-Jones {sigma, eps, -},                      */
/* 1 = Morse {D, alpha, r0}, 2 = soft sphere {sigma, eps, alpha}.            */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t kind;
  int32_t shift;   /* 1: subtract phi(rc) from every pair energy           */
  double p[3];
  double rc;       /* pair cutoff; soft sphere uses rc = sigma             */
} or_pot;

/* phi, dphi/dr, d2phi/dr2 of the unshifted pair potential at distance r.
 * LJ:    phi = 4 eps [(s/r)^12 - (s/r)^6]
 * Morse: phi = D [exp(-2a(r-r0)) - 2 exp(-a(r-r0))]
 * SS:    phi = (eps/alpha) (1 - r/sigma)^alpha for r < sigma, else 0
 * Pinned by: dimer minima (LJ -eps at 2^(1/6) sigma, Morse -D at r0),
 * soft-sphere end values, central differences of phi and dphi. */
static void pot_eval(const or_pot* P, double r, double* phi, double* d1, double* d2) {
  if (P->kind == 0) {
    double sg = P->p[0], ep = P->p[1];
    double s = sg / r, s6 = s * s * s * s * s * s, s12 = s6 * s6;
    *phi = 4.0 * ep * (s12 - s6);
    *d1 = -24.0 * ep / r * (2.0 * s12 - s6);
    *d2 = 24.0 * ep / (r * r) * (26.0 * s12 - 7.0 * s6);
  } else if (P->kind == 1) {
    double D = P->p[0], a = P->p[1], r0 = P->p[2];
    double e = exp(-a * (r - r0));
    *phi = D * (e * e - 2.0 * e);
    *d1 = 2.0 * a * D * (e - e * e);
    *d2 = 2.0 * a * a * D * (2.0 * e * e - e);
  } else {
    double sg = P->p[0], ep = P->p[1], al = P->p[2];
    if (r >= sg) { *phi = 0; *d1 = 0; *d2 = 0; return; }
    double t = 1.0 - r / sg;
    *phi = ep / al * pow(t, al);
    *d1 = -ep / sg * pow(t, al - 1.0);
    *d2 = ep / (sg * sg) * (al - 1.0) * pow(t, al - 2.0);
  }
}

static double pot_cutoff(const or_pot* P) { return P->kind == 2 ? P->p[0] : P->rc; }

/* Derivatives of phi and dphi/dr with respect to the three parameters p[k],
 * at fixed r and fixed numeric cutoff.  Pinned by central differences in p. */
static void pot_param_grad(const or_pot* P, double r, double dphi[3], double dd1[3]) {
  dphi[0] = dphi[1] = dphi[2] = 0; dd1[0] = dd1[1] = dd1[2] = 0;
  if (P->kind == 0) {
    double sg = P->p[0], ep = P->p[1];
    double s = sg / r, s6 = s * s * s * s * s * s, s12 = s6 * s6;
    dphi[0] = 24.0 * ep / sg * (2.0 * s12 - s6);          /* d phi / d sigma */
    dphi[1] = 4.0 * (s12 - s6);                           /* d phi / d eps   */
    dd1[0] = -144.0 * ep / (r * sg) * (4.0 * s12 - s6);   /* d phi' / d sigma */
    dd1[1] = -24.0 / r * (2.0 * s12 - s6);                /* d phi' / d eps   */
  } else if (P->kind == 1) {
    double D = P->p[0], a = P->p[1], r0 = P->p[2];
    double e = exp(-a * (r - r0)), x = r - r0;
    dphi[0] = e * e - 2.0 * e;
    dphi[1] = 2.0 * D * x * (e - e * e);
    dphi[2] = 2.0 * a * D * (e * e - e);
    dd1[0] = 2.0 * a * (e - e * e);
    dd1[1] = 2.0 * D * (e - e * e) + 2.0 * a * D * x * (2.0 * e * e - e);
    dd1[2] = -2.0 * a * a * D * (2.0 * e * e - e);
  } else {
    double sg = P->p[0], ep = P->p[1], al = P->p[2];
    if (r >= sg) return;
    double t = 1.0 - r / sg, lt = log(t);
    double ta = pow(t, al), ta1 = pow(t, al - 1.0), ta2 = pow(t, al - 2.0);
    dphi[0] = ep * ta1 * r / (sg * sg);
    dphi[1] = ta / al;
    dphi[2] = -ep / (al * al) * ta + ep / al * ta * lt;
    dd1[0] = ep / (sg * sg) * ta1 - ep / sg * (al - 1.0) * ta2 * r / (sg * sg);
    dd1[1] = -ta1 / sg;
    dd1[2] = -ep / sg * ta1 * lt;
  }
}

/* ------------------------------------------------------------------------- */
/* Cell geometry (rows = lattice vectors).                                   */
/* ------------------------------------------------------------------------- */
static double det3(const double* h) {
  return h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
         h[2] * (h[3] * h[7] - h[4] * h[6]);
}
static void inv3(const double* h, double* g) {
  double d = det3(h);
  g[0] = (h[4] * h[8] - h[5] * h[7]) / d; g[1] = (h[2] * h[7] - h[1] * h[8]) / d;
  g[2] = (h[1] * h[5] - h[2] * h[4]) / d; g[3] = (h[5] * h[6] - h[3] * h[8]) / d;
  g[4] = (h[0] * h[8] - h[2] * h[6]) / d; g[5] = (h[2] * h[3] - h[0] * h[5]) / d;
  g[6] = (h[3] * h[7] - h[4] * h[6]) / d; g[7] = (h[1] * h[6] - h[0] * h[7]) / d;
  g[8] = (h[0] * h[4] - h[1] * h[3]) / d;
}
/* Perpendicular width of the cell along each lattice direction:
 * w_a = V / |h_b x h_c|.  A pair vector d = (ds) h satisfies |d| >= |ds_a| w_a. */
static void widths3(const double* h, double* w) {
  double V = fabs(det3(h));
  for (int a = 0; a < 3; a++) {
    const double* b = h + 3 * ((a + 1) % 3);
    const double* c = h + 3 * ((a + 2) % 3);
    double cx = b[1] * c[2] - b[2] * c[1], cy = b[2] * c[0] - b[0] * c[2], cz = b[0] * c[1] - b[1] * c[0];
    w[a] = V / sqrt(cx * cx + cy * cy + cz * cz);
  }
}
static void frac_of(const double* x, const double* g, double* s) {
  for (int a = 0; a < 3; a++) s[a] = x[0] * g[a] + x[1] * g[3 + a] + x[2] * g[6 + a];
}

/* ------------------------------------------------------------------------- */
/* Neighbour set, by definition (multi-image brute force).                   */
/* N(s) = {(i, j, n): i, j in s, n integer on periodic axes, (i,n) != (j,0),  */
/*         |x_j + n h - x_i| < r}.                                           */
/* For every ordered (i, j) the images are enumerated over the exact bounds  */
/* n_a in [floor(-ds_a - r/w_a), ceil(-ds_a + r/w_a)] (ds = s_j - s_i,       */
/* unwrapped), which contain every image with |d| < r since |d| >= |ds_a +   */
/* n_a| w_a.  Pinned by: the cell-list enumeration below, FCC shell counts. */
/* ------------------------------------------------------------------------- */
typedef void (*pair_cb)(void* ctx, int i, int j, const int* n, const double* d, double r);

static void for_pairs_brute(int N, const double* x, const double* h, const uint8_t* pbc, double rmax,
                            pair_cb cb, void* ctx) {
  double g[9], w[3];
  inv3(h, g); widths3(h, w);
  double* s = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
  for (int i = 0; i < N; i++) frac_of(x + 3 * i, g, s + 3 * i);
  for (int i = 0; i < N; i++) {
    for (int j = 0; j < N; j++) {
      double ds[3]; int lo[3], hi[3];
      for (int a = 0; a < 3; a++) {
        ds[a] = s[3 * j + a] - s[3 * i + a];
        if (pbc[a]) { lo[a] = (int)floor(-ds[a] - rmax / w[a]); hi[a] = (int)ceil(-ds[a] + rmax / w[a]); }
        else { lo[a] = hi[a] = 0; }
      }
      int n[3];
      for (n[0] = lo[0]; n[0] <= hi[0]; n[0]++)
        for (n[1] = lo[1]; n[1] <= hi[1]; n[1]++)
          for (n[2] = lo[2]; n[2] <= hi[2]; n[2]++) {
            if (i == j && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
            double d[3];
            for (int c = 0; c < 3; c++)
              d[c] = x[3 * j + c] - x[3 * i + c] + n[0] * h[c] + n[1] * h[3 + c] + n[2] * h[6 + c];
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r < rmax) cb(ctx, i, j, n, d, r);
          }
    }
  }
  free(s);
}

/* Cell-list enumeration of the same set (used for timing large inputs).
 * Bins per axis n_a = max(1, floor(w_a / r)); fractional coordinates are
 * wrapped to [0,1) for binning only; each atom visits the bins k-m..k+m with
 * m_a = ceil(r n_a / w_a), mapping out-of-range bins back with an image
 * shift.  The reported n is the image relative to the unwrapped input
 * positions, so the output equals the brute-force set.  Periodic axes only. */
static void for_pairs_cells(int N, const double* x, const double* h, double rmax, pair_cb cb, void* ctx) {
  double g[9], w[3];
  inv3(h, g); widths3(h, w);
  int nb[3], m[3];
  for (int a = 0; a < 3; a++) {
    nb[a] = (int)floor(w[a] / rmax); if (nb[a] < 1) nb[a] = 1;
    if (nb[a] > 256) nb[a] = 256;
    m[a] = (int)ceil(rmax * nb[a] / w[a]); if (m[a] < 1) m[a] = 1;
  }
  int nc = nb[0] * nb[1] * nb[2];
  double* sw = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
  int* fl = (int*)malloc(sizeof(int) * 3 * (N > 0 ? N : 1));
  int* cell = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
  int* head = (int*)malloc(sizeof(int) * (nc + 1));
  int* list = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
  for (int i = 0; i < N; i++) {
    double s[3]; frac_of(x + 3 * i, g, s);
    int k[3];
    for (int a = 0; a < 3; a++) {
      double f = floor(s[a]);
      fl[3 * i + a] = (int)f; sw[3 * i + a] = s[a] - f;
      k[a] = (int)(sw[3 * i + a] * nb[a]); if (k[a] >= nb[a]) k[a] = nb[a] - 1; if (k[a] < 0) k[a] = 0;
    }
    cell[i] = (k[2] * nb[1] + k[1]) * nb[0] + k[0];
  }
  for (int c = 0; c <= nc; c++) head[c] = 0;
  for (int i = 0; i < N; i++) head[cell[i] + 1]++;
  for (int c = 0; c < nc; c++) head[c + 1] += head[c];
  { int* fill = (int*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int));
    for (int i = 0; i < N; i++) list[head[cell[i]] + fill[cell[i]]++] = i;
    free(fill); }
  for (int i = 0; i < N; i++) {
    int ci = cell[i], k[3] = {ci % nb[0], (ci / nb[0]) % nb[1], ci / (nb[0] * nb[1])};
    for (int dz = -m[2]; dz <= m[2]; dz++)
      for (int dy = -m[1]; dy <= m[1]; dy++)
        for (int dx = -m[0]; dx <= m[0]; dx++) {
          int kk[3] = {k[0] + dx, k[1] + dy, k[2] + dz}, img[3], cc[3];
          for (int a = 0; a < 3; a++) {
            img[a] = (int)floor((double)kk[a] / nb[a]);
            cc[a] = kk[a] - img[a] * nb[a];
          }
          int c2 = (cc[2] * nb[1] + cc[1]) * nb[0] + cc[0];
          for (int q = head[c2]; q < head[c2 + 1]; q++) {
            int j = list[q];
            if (j == i && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
            double ds[3];
            for (int a = 0; a < 3; a++) ds[a] = sw[3 * j + a] + img[a] - sw[3 * i + a];
            double d[3];
            for (int c = 0; c < 3; c++) d[c] = ds[0] * h[c] + ds[1] * h[3 + c] + ds[2] * h[6 + c];
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r < rmax) {
              int n[3];
              for (int a = 0; a < 3; a++) n[a] = img[a] - fl[3 * j + a] + fl[3 * i + a];
              /* d recomputed from the unwrapped inputs with the original image */
              for (int c = 0; c < 3; c++)
                d[c] = x[3 * j + c] - x[3 * i + c] + n[0] * h[c] + n[1] * h[3 + c] + n[2] * h[6 + c];
              r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
              if (r < rmax) cb(ctx, i, j, n, d, r);
            }
          }
        }
  }
  free(sw); free(fl); free(cell); free(head); free(list);
}

static void for_pairs(int use_cells, int N, const double* x, const double* h, const uint8_t* pbc, double rmax,
                      pair_cb cb, void* ctx) {
  if (use_cells && pbc[0] && pbc[1] && pbc[2]) for_pairs_cells(N, x, h, rmax, cb, ctx);
  else for_pairs_brute(N, x, h, pbc, rmax, cb, ctx);
}

/* Public: list the neighbour triples (i, j, n) of one system.  Returns the
 * number of pairs; writes at most cap of them. */
typedef struct { int64_t cnt, cap; int32_t* out; } list_ctx;
static void list_cb(void* c_, int i, int j, const int* n, const double* d, double r) {
  (void)d; (void)r;
  list_ctx* c = (list_ctx*)c_;
  if (c->cnt < c->cap) {
    int32_t* o = c->out + 5 * c->cnt;
    o[0] = i; o[1] = j; o[2] = n[0]; o[3] = n[1]; o[4] = n[2];
  }
  c->cnt++;
}
int64_t or_neighbors(int N, const double* x, const double* h, const uint8_t* pbc, double rmax, int use_cells,
                     int32_t* out /*[cap,5]*/, int64_t cap) {
  list_ctx c = {0, cap, out};
  for_pairs(use_cells, N, x, h, pbc, rmax, list_cb, &c);
  return c.cnt;
}

/* ------------------------------------------------------------------------- */
/* Energy, forces, stress (Sec. 2 output schema: energies, forces, stress).  */
/* E = 1/2 sum_{(i,j,n) in N, r<rc} [phi(r) - phi_c]                          */
/* F_i = sum_{(j,n)} phi'(r) d/r,  d = x_j + n h - x_i                        */
/* stress = (1/V) 1/2 sum phi'(r) d (x) d / r   (= (1/V) dE/d strain; ASE sign) */
/* Pinned by: dimer closed forms, FCC lattice sums, Newton's third law,      */
/* central differences of E in x and in strain, PyTorch FP64 autograd.       */
/* ------------------------------------------------------------------------- */
typedef struct { const or_pot* P; double phic; double E; double* F; double W[9]; double* e_atom; } force_ctx;
static void force_cb(void* c_, int i, int j, const int* n, const double* d, double r) {
  (void)j; (void)n;
  force_ctx* c = (force_ctx*)c_;
  double phi, d1, d2;
  pot_eval(c->P, r, &phi, &d1, &d2);
  double e = 0.5 * (phi - c->phic);
  c->E += e;
  if (c->e_atom) c->e_atom[i] += e;
  for (int a = 0; a < 3; a++) c->F[3 * i + a] += d1 * d[a] / r;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) c->W[3 * a + b] += 0.5 * d1 * d[a] * d[b] / r;
}

static double pot_shift(const or_pot* P) {
  if (!P->shift || P->kind == 2) return 0.0;
  double phi, d1, d2; pot_eval(P, P->rc, &phi, &d1, &d2);
  return phi;
}

/* Batched: offsets[B+1] delimit each system's atoms in the concatenated
 * arrays (Sec. 3: atom-wise arrays concatenated, system-wise stacked). */
void or_forces(int B, const int64_t* offsets, const double* x, const double* cells, const uint8_t* pbc,
               const int32_t* pot_of_sys, const or_pot* pots, int use_cells,
               double* E, double* F, double* stress, double* e_atom) {
  int64_t N = offsets[B];
  memset(F, 0, sizeof(double) * 3 * N);
  if (e_atom) memset(e_atom, 0, sizeof(double) * N);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const or_pot* P = pots + pot_of_sys[s];
    force_ctx c = {P, pot_shift(P), 0.0, F + 3 * o, {0}, e_atom ? e_atom + o : NULL};
    for_pairs(use_cells, n, x + 3 * o, cells + 9 * s, pbc + 3 * s, pot_cutoff(P), force_cb, &c);
    E[s] = c.E;
    double V = fabs(det3(cells + 9 * s));
    if (stress) for (int k = 0; k < 9; k++) stress[9 * s + k] = c.W[k] / V;
  }
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of            */
/* (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2, c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0),*/
/* key bumped by the Weyl constants between rounds.                          */
/* Pinned by the published known-answer vectors.                             */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three N(0,1) draws for one atom at one step.  Counter = (step, local atom
 * index, 0, 0); key = (seed, system uid).  Uniforms u = (k + 1/2) 2^-32 in
 * (0,1); Box-Muller: z0 = R cos(2 pi u1), z1 = R sin(2 pi u1) with
 * R = sqrt(-2 ln u0) from words (0,1); z2 = sqrt(-2 ln u2) cos(2 pi u3). */
void or_normals3(uint64_t step, uint32_t local_atom, uint32_t seed, uint32_t uid, double z[3]) {
  uint32_t ctr[4] = {(uint32_t)step, local_atom, (uint32_t)(step >> 32), 0u}, key[2] = {seed, uid}, o[4];
  or_philox4x32_10(ctr, key, o);
  const double two_pi = 6.283185307179586476925286766559;
  double u0 = ((double)o[0] + 0.5) * 2.3283064365386962890625e-10;
  double u1 = ((double)o[1] + 0.5) * 2.3283064365386962890625e-10;
  double u2 = ((double)o[2] + 0.5) * 2.3283064365386962890625e-10;
  double u3 = ((double)o[3] + 0.5) * 2.3283064365386962890625e-10;
  double R0 = sqrt(-2.0 * log(u0)), R1 = sqrt(-2.0 * log(u2));
  z[0] = R0 * cos(two_pi * u1);
  z[1] = R0 * sin(two_pi * u1);
  z[2] = R1 * cos(two_pi * u3);
}

/* ------------------------------------------------------------------------- */
/* Molecular dynamics (Sec. 4 runs Langevin MD; NVE velocity Verlet is the   */
/* gamma -> 0, noise-free limit).                                            */
/* ------------------------------------------------------------------------- */
static double kinetic(int64_t o, int n, const double* v, const double* m) {
  double k = 0;
  for (int i = 0; i < n; i++)
    k += 0.5 * m[o + i] * (v[3 * (o + i)] * v[3 * (o + i)] + v[3 * (o + i) + 1] * v[3 * (o + i) + 1] +
                           v[3 * (o + i) + 2] * v[3 * (o + i) + 2]);
  return k;
}

/* One system's forces into F (scratch), energy returned. */
static double sys_forces(int use_cells, int n, const double* x, const double* h, const uint8_t* pbc,
                         const or_pot* P, double* F) {
  memset(F, 0, sizeof(double) * 3 * n);
  force_ctx c = {P, pot_shift(P), 0.0, F, {0}, NULL};
  for_pairs(use_cells, n, x, h, pbc, pot_cutoff(P), force_cb, &c);
  return c.E;
}

/* Velocity Verlet, n_steps:
 *   v <- v + dt/(2m) F;  x <- x + dt v;  F <- F(x);  v <- v + dt/(2m) F.
 * Langevin (kind 1): BAOAB -- B half kick, A half drift, O exact OU step
 *   v <- c1 v + sqrt((1 - c1^2) kT/m) xi, c1 = exp(-gamma dt),
 * A half drift, new forces, B half kick.  xi from or_normals3 with counter
 * step = step0 + k (k = 0..n_steps-1), local atom index within the system,
 * key (seed, uid[s]).  Positions are not wrapped.
 * Outputs: E_pot[B], KE[B] after the last step.
 * Pinned by: time reversibility (VV), energy drift, <KE> = (3N-3)/2 kT
 * equipartition (BAOAB), gamma -> 0 reducing BAOAB to VV. */
void or_md(int B, const int64_t* offsets, double* x, double* v, const double* mass, const double* cells,
           const uint8_t* pbc, const int32_t* pot_of_sys, const or_pot* pots, int use_cells,
           int kind, double dt, int n_steps, const double* kT, double gamma, uint32_t seed,
           const uint32_t* uid, uint64_t step0, double* E_pot, double* KE) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const or_pot* P = pots + pot_of_sys[s];
    const double* h = cells + 9 * s;
    double* xs = x + 3 * o; double* vs = v + 3 * o;
    double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double E = sys_forces(use_cells, n, xs, h, pbc + 3 * s, P, F);
    double c1 = exp(-gamma * dt);
    for (int k = 0; k < n_steps; k++) {
      for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) vs[3 * i + a] += 0.5 * dt / mass[o + i] * F[3 * i + a];
      if (kind == 0) {
        for (int i = 0; i < 3 * n; i++) xs[i] += dt * vs[i];
      } else {
        for (int i = 0; i < 3 * n; i++) xs[i] += 0.5 * dt * vs[i];
        for (int i = 0; i < n; i++) {
          double z[3];
          or_normals3(step0 + (uint64_t)k, (uint32_t)i, seed, uid[s], z);
          double sc = sqrt((1.0 - c1 * c1) * kT[s] / mass[o + i]);
          for (int a = 0; a < 3; a++) vs[3 * i + a] = c1 * vs[3 * i + a] + sc * z[a];
        }
        for (int i = 0; i < 3 * n; i++) xs[i] += 0.5 * dt * vs[i];
      }
      E = sys_forces(use_cells, n, xs, h, pbc + 3 * s, P, F);
      for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) vs[3 * i + a] += 0.5 * dt / mass[o + i] * F[3 * i + a];
    }
    if (E_pot) E_pot[s] = E;
    if (KE) KE[s] = kinetic(o, n, v, mass);
    free(F);
  }
}

/* ------------------------------------------------------------------------- */
/* NVT with a Nose-Hoover chain (one of the integrators the paper lists,      */
/* Sec. 1; chain of Martyna, Klein and Tuckerman 1992, time-reversible       */
/* factorisation of Martyna, Tuckerman, Tobias and Klein 1996 with a single  */
/* sub-step).  One step:                                                      */
/*   C(dt/2); v += dt/(2m) F; x += dt v; F = F(x); v += dt/(2m) F; C(dt/2).   */
/* Chain of M = 3 thermostats per system with positions xi_k and velocities  */
/* w_k; masses Q_1 = Nf kT tau^2, Q_k = kT tau^2 (k > 1); Nf = 3N - 3 (the    */
/* total momentum stays zero).  Forces on the chain: G_1 = (2K - Nf kT)/Q_1, */
/* G_k = (Q_{k-1} w_{k-1}^2 - kT)/Q_k, with K the kinetic energy.  C(h):     */
/*   w_M += h/2 G_M;                                                          */
/*   for k = M-1 .. 1: w_k *= e^{-h/4 w_{k+1}}; w_k += h/2 G_k;               */
/*                     w_k *= e^{-h/4 w_{k+1}};                               */
/*   xi_k += h w_k (all k); atoms: v *= e^{-h w_1} (K *= e^{-2 h w_1});       */
/*   for k = 1 .. M-1: w_k *= e^{-h/4 w_{k+1}}; w_k += h/2 G_k (current K or  */
/*                     w_{k-1}); w_k *= e^{-h/4 w_{k+1}};                     */
/*   w_M += h/2 G_M.                                                          */
/* Conserved: K + U + sum_k Q_k w_k^2/2 + Nf kT xi_1 + kT sum_{k>1} xi_k.     */
/* Pinned by: the conserved quantity; an inert chain (tau -> inf) reproduces  */
/* velocity Verlet; time reversibility; <K> = Nf kT/2 on a long run.          */
/* ------------------------------------------------------------------------- */
#define OR_NHC_M 3
static double nhc_half(double h, double K, double nf, double kT, double tau, double* st) {
  double* xi = st; double* w = st + OR_NHC_M;
  double Q[OR_NHC_M];
  Q[0] = nf * kT * tau * tau;
  for (int k = 1; k < OR_NHC_M; k++) Q[k] = kT * tau * tau;
  const int M = OR_NHC_M;
  double G = (Q[M - 2] * w[M - 2] * w[M - 2] - kT) / Q[M - 1];
  w[M - 1] += 0.5 * h * G;
  for (int k = M - 2; k >= 0; k--) {
    double e = exp(-0.25 * h * w[k + 1]);
    w[k] *= e;
    G = k == 0 ? (2.0 * K - nf * kT) / Q[0] : (Q[k - 1] * w[k - 1] * w[k - 1] - kT) / Q[k];
    w[k] += 0.5 * h * G;
    w[k] *= e;
  }
  for (int k = 0; k < M; k++) xi[k] += h * w[k];
  double scale = exp(-h * w[0]);
  K *= scale * scale;
  for (int k = 0; k < M - 1; k++) {
    double e = exp(-0.25 * h * w[k + 1]);
    w[k] *= e;
    G = k == 0 ? (2.0 * K - nf * kT) / Q[0] : (Q[k - 1] * w[k - 1] * w[k - 1] - kT) / Q[k];
    w[k] += 0.5 * h * G;
    w[k] *= e;
  }
  G = (Q[M - 2] * w[M - 2] * w[M - 2] - kT) / Q[M - 1];
  w[M - 1] += 0.5 * h * G;
  return scale;
}

/* n_steps of NVT-NHC; nhc [B][2M] (xi_1..M, w_1..M) is read and updated;    */
/* H_ext [B] (may be NULL) receives the conserved quantity at the end.        */
void or_md_nhc(int B, const int64_t* offsets, double* x, double* v, const double* mass, const double* cells,
               const uint8_t* pbc, const int32_t* pot_of_sys, const or_pot* pots, int use_cells, double dt,
               int n_steps, const double* kT, double tau, double* nhc, double* E_pot, double* KE, double* H_ext) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const or_pot* P = pots + pot_of_sys[s];
    const double* h = cells + 9 * s;
    double* xs = x + 3 * o; double* vs = v + 3 * o;
    double* st = nhc + 2 * OR_NHC_M * s;
    const double nf = 3.0 * n - 3.0 > 1.0 ? 3.0 * n - 3.0 : 1.0;
    double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double E = sys_forces(use_cells, n, xs, h, pbc + 3 * s, P, F);
    for (int k = 0; k < n_steps; k++) {
      double sc = nhc_half(0.5 * dt, kinetic(o, n, v, mass), nf, kT[s], tau, st);
      for (int i = 0; i < 3 * n; i++) vs[i] *= sc;
      for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) vs[3 * i + a] += 0.5 * dt / mass[o + i] * F[3 * i + a];
      for (int i = 0; i < 3 * n; i++) xs[i] += dt * vs[i];
      E = sys_forces(use_cells, n, xs, h, pbc + 3 * s, P, F);
      for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) vs[3 * i + a] += 0.5 * dt / mass[o + i] * F[3 * i + a];
      sc = nhc_half(0.5 * dt, kinetic(o, n, v, mass), nf, kT[s], tau, st);
      for (int i = 0; i < 3 * n; i++) vs[i] *= sc;
    }
    double K = kinetic(o, n, v, mass);
    if (E_pot) E_pot[s] = E;
    if (KE) KE[s] = K;
    if (H_ext) {
      double Q1 = nf * kT[s] * tau * tau, Qk = kT[s] * tau * tau;
      double He = K + E + 0.5 * Q1 * st[OR_NHC_M] * st[OR_NHC_M] + nf * kT[s] * st[0];
      for (int k = 1; k < OR_NHC_M; k++) He += 0.5 * Qk * st[OR_NHC_M + k] * st[OR_NHC_M + k] + kT[s] * st[k];
      H_ext[s] = He;
    }
    free(F);
  }
}

/* ------------------------------------------------------------------------- */
/* NPT: isotropic barostat of Martyna, Tobias and Klein (1994) with Langevin  */
/* (Ornstein-Uhlenbeck) friction and noise on the atoms and on the piston;   */
/* the paper lists NPT among its integrators (Sec. 1) without a scheme.       */
/* Per system: piston velocity v_e (the cell scales isotropically,            */
/* dh/dt = v_e h), piston mass W = (Nf + 3) kT tau^2, Nf = 3N, a = 1 + 3/Nf. */
/* Without friction:                                                          */
/*   dx/dt = v + v_e x,   dv/dt = F/m - a v_e v,   dh/dt = v_e h,            */
/*   W dv_e/dt = a 2K + Xi - 3 V P_ext,                                       */
/* with K the kinetic energy, V = |det h| and Xi = -sum_pairs phi'(r) r the  */
/* pair virial (= -tr of the stress accumulator W_ab = 1/2 sum phi' d d / r). */
/* It conserves H = K + U + W v_e^2 / 2 + P_ext V.                            */
/* One step, each sub-flow solved exactly (symmetric, as in the MTK           */
/* integrator of Tuckerman et al. 2006, with BAOAB's O in the middle):        */
/*   Be(dt/2): v_e += dt/2 (a 2K + Xi - 3 V P_ext) / W                       */
/*   B(dt/2):  v <- v e^{-c dt/2} + dt/2 e^{-c dt/4} shc(c dt/4) F/m, c = a v_e */
/*   A(dt/2):  x <- x e^{v_e dt/2} + dt/2 e^{v_e dt/4} shc(v_e dt/4) v;       */
/*             h <- h e^{v_e dt/2}                                            */
/*   O(dt):    v <- c1 v + sqrt((1 - c1^2) kT/m) xi_i,                        */
/*             v_e <- c1 v_e + sqrt((1 - c1^2) kT/W) xi_e,  c1 = e^{-gamma dt} */
/*   A(dt/2); forces, U and Xi at the new x and h; B(dt/2); Be(dt/2).         */
/* shc(y) = sinh(y)/y.  xi_i = or_normals3(step, i, seed, uid); xi_e = the    */
/* first normal of or_normals3(step, 0xffffffff, seed, uid).                  */
/* Pinned by: the conserved H without friction (and its O(dt^2) size),        */
/* time reversibility, an inert piston (tau -> inf) reproducing BAOAB, and   */
/* the lattice constant of a cold damped FCC crystal against the minimum of  */
/* the independent lattice sum's enthalpy u(a) + P_ext a^3/4.                */
/* ------------------------------------------------------------------------- */
static double shc(double y) {
  if (fabs(y) < 1e-3) { double y2 = y * y; return 1.0 + y2 / 6.0 * (1.0 + y2 / 20.0); }
  return sinh(y) / y;
}

/* One system's forces into F, energy returned, pair virial Xi into *xi. */
static double sys_forces_virial(int use_cells, int n, const double* x, const double* h, const uint8_t* pbc,
                                const or_pot* P, double* F, double* xi) {
  memset(F, 0, sizeof(double) * 3 * n);
  force_ctx c = {P, pot_shift(P), 0.0, F, {0}, NULL};
  for_pairs(use_cells, n, x, h, pbc, pot_cutoff(P), force_cb, &c);
  *xi = -(c.W[0] + c.W[4] + c.W[8]);
  return c.E;
}

/* n_steps of NPT per system; cells [B][9] and baro [B] (v_e) are read and   */
/* updated.  Outputs after the last step: E_pot, KE, H_ext (the quantity     */
/* conserved without friction) and P_inst = (2K + Xi)/(3V) (may be NULL).    */
void or_md_npt(int B, const int64_t* offsets, double* x, double* v, const double* mass, double* cells,
               const uint8_t* pbc, const int32_t* pot_of_sys, const or_pot* pots, int use_cells, double dt,
               int n_steps, const double* kT, double gamma, double tau, double p_ext, uint32_t seed,
               const uint32_t* uid, uint64_t step0, double* baro, double* E_pot, double* KE, double* H_ext,
               double* P_inst) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const or_pot* P = pots + pot_of_sys[s];
    double* h = cells + 9 * s;
    double* xs = x + 3 * o; double* vs = v + 3 * o;
    const double nf = 3.0 * n, al = 1.0 + 3.0 / nf;
    const double Wp = (nf + 3.0) * kT[s] * tau * tau;
    const double c1 = exp(-gamma * dt);
    double ve = baro[s];
    double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double xi;
    double E = sys_forces_virial(use_cells, n, xs, h, pbc + 3 * s, P, F, &xi);
    for (int k = 0; k < n_steps; k++) {
      double V = fabs(det3(h));
      ve += 0.5 * dt * (al * 2.0 * kinetic(o, n, v, mass) + xi - 3.0 * V * p_ext) / Wp;   /* Be */
      double c = al * ve;                                                                  /* B */
      double eb = exp(-0.5 * c * dt), fb = 0.5 * dt * exp(-0.25 * c * dt) * shc(0.25 * c * dt);
      for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) vs[3 * i + a] = vs[3 * i + a] * eb + fb * F[3 * i + a] / mass[o + i];
      for (int half = 0; half < 2; half++) {                                               /* A O A */
        if (half == 1) {
          for (int i = 0; i < n; i++) {
            double z[3];
            or_normals3(step0 + (uint64_t)k, (uint32_t)i, seed, uid[s], z);
            double sc = sqrt((1.0 - c1 * c1) * kT[s] / mass[o + i]);
            for (int a = 0; a < 3; a++) vs[3 * i + a] = c1 * vs[3 * i + a] + sc * z[a];
          }
          double z[3];
          or_normals3(step0 + (uint64_t)k, 0xffffffffu, seed, uid[s], z);
          ve = c1 * ve + sqrt((1.0 - c1 * c1) * kT[s] / Wp) * z[0];
        }
        double ea = exp(0.5 * ve * dt), fa = 0.5 * dt * exp(0.25 * ve * dt) * shc(0.25 * ve * dt);
        for (int i = 0; i < 3 * n; i++) xs[i] = xs[i] * ea + fa * vs[i];
        for (int q = 0; q < 9; q++) h[q] *= ea;
      }
      E = sys_forces_virial(use_cells, n, xs, h, pbc + 3 * s, P, F, &xi);
      c = al * ve;                                                                         /* B */
      eb = exp(-0.5 * c * dt); fb = 0.5 * dt * exp(-0.25 * c * dt) * shc(0.25 * c * dt);
      for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) vs[3 * i + a] = vs[3 * i + a] * eb + fb * F[3 * i + a] / mass[o + i];
      V = fabs(det3(h));
      ve += 0.5 * dt * (al * 2.0 * kinetic(o, n, v, mass) + xi - 3.0 * V * p_ext) / Wp;   /* Be */
    }
    double K = kinetic(o, n, v, mass), V = fabs(det3(h));
    baro[s] = ve;
    if (E_pot) E_pot[s] = E;
    if (KE) KE[s] = K;
    if (H_ext) H_ext[s] = K + E + 0.5 * Wp * ve * ve + p_ext * V;
    if (P_inst) P_inst[s] = (2.0 * K + xi) / (3.0 * V);
    free(F);
  }
}

/* ------------------------------------------------------------------------- */
/* Variable-cell FIRE (Bitzek et al. 2006; the paper's "structural relaxation */
/* optimizers", Sec. 1, run under in-flight batching, Sec. 3).               */
/* Generalised coordinates per system: xt_i = x_i Fd^-T (N rows) and the cell */
/* block Q = c Fd (c = N atoms), with h = h0 Fd^T and x = xt Fd^T.           */
/* Generalised forces: ft_i = F_i Fd, G = -V (sigma + p I) Fd^-T / c.        */
/* Per step (unit masses): P = f.v over all DOF; if P > 0: v <- (1-a) v +    */
/* a |v| f/|f|, and if Npos > Nmin: dt <- min(dt finc, dtmax), a <- a fa;    */
/* Npos++.  Else v <- 0, dt <- dt fdec, a <- a0, Npos <- 0.  The first step   */
/* of a system skips this test.  Then v <- v + dt f, dq = dt v clamped to    */
/* |dq| <= maxstep (whole system vector), q <- q + dq.                       */
/* Convergence (tested on the forces and stress at the current q, before the */
/* update): max_i |F_i| <= fmax and max_ab |sigma_ab| <= smax; converged     */
/* systems are frozen.                                                       */
/* Pinned by: the relaxed FCC lattice constant against an independent lattice */
/* sum minimisation, and the stress/force zero at convergence.               */
/* ------------------------------------------------------------------------- */
typedef struct {
  double dt, alpha; int32_t npos; int32_t started; int32_t converged; int32_t nsteps;
  double Fd[9];   /* deformation gradient, row-major */
  double h0[9];   /* reference cell */
} or_fire_sys;

typedef struct {
  double dt_max, finc, fdec, alpha0, falpha, maxstep, fmax, smax, p_ext; int32_t nmin; int32_t variable_cell;
} or_fire_params;

static void mat_inv_T(const double* A, double* out) { /* out = A^-T */
  double g[9]; inv3(A, g);
  for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) out[3 * a + b] = g[3 * b + a];
}

/* x: physical positions [N,3] (updated); cells [B,9] (updated);
 * vel: generalised velocities [N + 3 per system rows, 3], laid out per system
 * as its N atom rows followed by its 3 cell rows (offset o + 3 s). */
void or_fire(int B, const int64_t* offsets, double* x, double* cells, const uint8_t* pbc,
             const int32_t* pot_of_sys, const or_pot* pots, int use_cells, or_fire_sys* st, double* vel,
             const or_fire_params* prm, int n_steps, double* E_out, double* fmax_out, double* smax_out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const or_pot* P = pots + pot_of_sys[s];
    or_fire_sys* S = st + s;
    double* xs = x + 3 * o; double* h = cells + 9 * s;
    double* vs = vel + 3 * (o + 3 * s);   /* n + 3 rows */
    int nd = n + 3;
    double* F = (double*)malloc(sizeof(double) * 3 * n);
    double* f = (double*)malloc(sizeof(double) * 3 * nd);
    double E = 0, fm = 0, sm = 0;
    double c = (double)n;
    for (int k = 0; k <= n_steps; k++) {
      /* forces and stress at the current configuration */
      memset(F, 0, sizeof(double) * 3 * n);
      force_ctx fc = {P, pot_shift(P), 0.0, F, {0}, NULL};
      for_pairs(use_cells, n, xs, h, pbc + 3 * s, pot_cutoff(P), force_cb, &fc);
      E = fc.E;
      double V = fabs(det3(h)), sig[9];
      for (int q = 0; q < 9; q++) sig[q] = fc.W[q] / V;
      fm = 0; sm = 0;
      for (int i = 0; i < n; i++) {
        double f2 = F[3 * i] * F[3 * i] + F[3 * i + 1] * F[3 * i + 1] + F[3 * i + 2] * F[3 * i + 2];
        if (sqrt(f2) > fm) fm = sqrt(f2);
      }
      for (int q = 0; q < 9; q++) if (fabs(sig[q]) > sm) sm = fabs(sig[q]);
      if (k == n_steps) break;  /* final evaluation only (reported values) */
      if (S->converged) continue;
      if (fm <= prm->fmax && (!prm->variable_cell || sm <= prm->smax)) { S->converged = 1; continue; }
      /* generalised forces */
      const double* Fd = S->Fd;
      for (int i = 0; i < n; i++)
        for (int b = 0; b < 3; b++)
          f[3 * i + b] = F[3 * i] * Fd[0 * 3 + b] + F[3 * i + 1] * Fd[1 * 3 + b] + F[3 * i + 2] * Fd[2 * 3 + b];
      if (prm->variable_cell) {
        double FiT[9], sp[9];
        mat_inv_T(Fd, FiT);
        for (int q = 0; q < 9; q++) sp[q] = sig[q];
        sp[0] += prm->p_ext; sp[4] += prm->p_ext; sp[8] += prm->p_ext;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) {
            double acc = 0;
            for (int q = 0; q < 3; q++) acc += sp[3 * a + q] * FiT[3 * q + b];
            f[3 * (n + a) + b] = -V * acc / c;
          }
      } else {
        for (int q = 0; q < 9; q++) f[3 * n + q] = 0;
      }
      /* FIRE velocity mixing / adaptation */
      if (S->started) {
        double Pw = 0, vv = 0, ff = 0;
        for (int q = 0; q < 3 * nd; q++) { Pw += f[q] * vs[q]; vv += vs[q] * vs[q]; ff += f[q] * f[q]; }
        if (Pw > 0) {
          double vn = sqrt(vv), fn = sqrt(ff);
          for (int q = 0; q < 3 * nd; q++) vs[q] = (1.0 - S->alpha) * vs[q] + S->alpha * vn * f[q] / fn;
          if (S->npos > prm->nmin) {
            S->dt = S->dt * prm->finc < prm->dt_max ? S->dt * prm->finc : prm->dt_max;
            S->alpha *= prm->falpha;
          }
          S->npos++;
        } else {
          for (int q = 0; q < 3 * nd; q++) vs[q] = 0;
          S->dt *= prm->fdec; S->alpha = prm->alpha0; S->npos = 0;
        }
      }
      S->started = 1;
      /* Euler step with the whole-vector step clamp */
      double dn = 0;
      for (int q = 0; q < 3 * nd; q++) { vs[q] += S->dt * f[q]; dn += (S->dt * vs[q]) * (S->dt * vs[q]); }
      dn = sqrt(dn);
      double scale = dn > prm->maxstep ? prm->maxstep / dn : 1.0;
      /* q <- q + dq: xt = x Fd^-T, Q = c Fd */
      double FiT[9]; mat_inv_T(Fd, FiT);
      double Fn[9];
      for (int q = 0; q < 9; q++) Fn[q] = Fd[q];
      if (prm->variable_cell)
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) Fn[3 * a + b] = (c * Fd[3 * a + b] + scale * S->dt * vs[3 * (n + a) + b]) / c;
      for (int i = 0; i < n; i++) {
        double xt[3];
        for (int b = 0; b < 3; b++)
          xt[b] = xs[3 * i] * FiT[b] + xs[3 * i + 1] * FiT[3 + b] + xs[3 * i + 2] * FiT[6 + b] +
                  scale * S->dt * vs[3 * i + b];
        /* x = xt Fn^T */
        for (int a = 0; a < 3; a++)
          xs[3 * i + a] = xt[0] * Fn[3 * a] + xt[1] * Fn[3 * a + 1] + xt[2] * Fn[3 * a + 2];
      }
      for (int q = 0; q < 9; q++) S->Fd[q] = Fn[q];
      /* h = h0 Fd^T */
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
          h[3 * a + b] = S->h0[3 * a] * Fn[3 * b] + S->h0[3 * a + 1] * Fn[3 * b + 1] + S->h0[3 * a + 2] * Fn[3 * b + 2];
      S->nsteps++;
    }
    if (E_out) E_out[s] = E;
    if (fmax_out) fmax_out[s] = fm;
    if (smax_out) smax_out[s] = sm;
    free(F); free(f);
  }
}

/* ------------------------------------------------------------------------- */
/* Pair-force adjoint (Sec. 2: gradients of a trajectory observable with     */
/* respect to model parameters).  For upstream gF [N,3], gE [B], gS [B,9]:   */
/*   gx_k = sum_{(j,n) in N(k)} K(d_kj) (gF_j - gF_k) - gE F_k               */
/*          - (1/V) sum_{(j,n)} dT(d_kj) : gS,                               */
/*   K(d) = phi'' dd^T/r^2 + (phi'/r)(I - dd^T/r^2),                          */
/*   T(d)_ab = (phi'/r) d_a d_b, dT/dd_c = ((phi''-phi'/r)/r^2) d_c d_a d_b   */
/*             + (phi'/r)(delta_ac d_b + d_a delta_bc);                      */
/*   gtheta_p = sum_(i,j,n) (dphi'/dp) (d/r).gF_i + gE 1/2 sum (dphi/dp -     */
/*             dphi_c/dp) + (1/2V) sum (dphi'/dp) d_a d_b / r gS_ab.          */
/* gtheta is accumulated per potential index.  Pinned by central differences */
/* of <gF, F> + gE E + <gS, sigma> in x and in the parameters.               */
/* ------------------------------------------------------------------------- */
typedef struct {
  const or_pot* P; const double* gF; double gE; const double* gS; double Vinv;
  double* gx; double gth[3]; double dphic[3];
} bwd_ctx;
static void bwd_cb(void* c_, int i, int j, const int* n, const double* d, double r) {
  (void)n;
  bwd_ctx* c = (bwd_ctx*)c_;
  double phi, d1, d2, dphi[3], dd1[3];
  pot_eval(c->P, r, &phi, &d1, &d2);
  pot_param_grad(c->P, r, dphi, dd1);
  double u[3] = {d[0] / r, d[1] / r, d[2] / r};
  double g[3] = {c->gF[3 * j] - c->gF[3 * i], c->gF[3 * j + 1] - c->gF[3 * i + 1], c->gF[3 * j + 2] - c->gF[3 * i + 2]};
  double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
  for (int a = 0; a < 3; a++) c->gx[3 * i + a] += d2 * ug * u[a] + d1 / r * (g[a] - ug * u[a]);
  double ugi = u[0] * c->gF[3 * i] + u[1] * c->gF[3 * i + 1] + u[2] * c->gF[3 * i + 2];
  for (int p = 0; p < 3; p++) c->gth[p] += dd1[p] * ugi + c->gE * 0.5 * (dphi[p] - c->dphic[p]);
  if (c->gS) {
    const double* S = c->gS;
    double A = (d2 - d1 / r) / (r * r), dSd = 0;
    for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) dSd += d[a] * S[3 * a + b] * d[b];
    for (int q = 0; q < 3; q++) {
      double Sd = 0, dS = 0;
      for (int b = 0; b < 3; b++) { Sd += S[3 * q + b] * d[b]; dS += d[b] * S[3 * b + q]; }
      /* d/dd_q of T:S, with d = x_j - x_i, so d/dx_i = -d/dd (and the mirror pair adds the same) */
      double dT = A * d[q] * dSd + d1 / r * (Sd + dS);
      c->gx[3 * i + q] -= c->Vinv * dT;
    }
    for (int p = 0; p < 3; p++) c->gth[p] += 0.5 * c->Vinv * dd1[p] / r * dSd;
  }
}
void or_forces_backward(int B, const int64_t* offsets, const double* x, const double* cells, const uint8_t* pbc,
                        const int32_t* pot_of_sys, const or_pot* pots, int n_pots, int use_cells,
                        const double* gF, const double* gE, const double* gS, double* gx, double* gth) {
  int64_t N = offsets[B];
  memset(gx, 0, sizeof(double) * 3 * N);
  double* part = (double*)calloc((size_t)B * 3, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const or_pot* P = pots + pot_of_sys[s];
    const double* h = cells + 9 * s;
    bwd_ctx c; memset(&c, 0, sizeof c);
    c.P = P; c.gF = gF + 3 * o; c.gE = gE ? gE[s] : 0.0; c.gS = gS ? gS + 9 * s : NULL;
    c.Vinv = 1.0 / fabs(det3(h)); c.gx = gx + 3 * o;
    if (P->shift && P->kind != 2) { double dd[3]; pot_param_grad(P, P->rc, c.dphic, dd); }
    for_pairs(use_cells, n, x + 3 * o, h, pbc + 3 * s, pot_cutoff(P), bwd_cb, &c);
    if (gE) {
      double* F = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
      sys_forces(use_cells, n, x + 3 * o, h, pbc + 3 * s, P, F);
      for (int i = 0; i < 3 * n; i++) gx[3 * o + i] -= gE[s] * F[i];
      free(F);
    }
    for (int p = 0; p < 3; p++) part[3 * s + p] = c.gth[p];
  }
  for (int q = 0; q < 3 * n_pots; q++) gth[q] = 0;
  for (int s = 0; s < B; s++)
    for (int p = 0; p < 3; p++) gth[3 * pot_of_sys[s] + p] += part[3 * s + p];
  free(part);
}

/* ------------------------------------------------------------------------- */
/* Gaussian-smeared radial distribution function (Sec. 2 observable).       */
/* K bins on [0, rmax): r_k = (k + 1/2) D, D = rmax/K, width w = D.          */
/* g_k = V/(N(N-1)) sum_{(i,j,n), r < rmax + 4w}                              */
/*        exp(-(r-r_k)^2/(2w^2)) / (sqrt(2 pi) w 4 pi r_k^2).                */
/* Pinned by: g -> 1 for uniform random points (ideal gas), and the          */
/* coordination-number integral of rho g 4 pi r^2 on an FCC lattice.        */
/* ------------------------------------------------------------------------- */
typedef struct { int K; double D, w, pref; double* g; const double* gg; double* gx; } rdf_ctx;
static void rdf_cb(void* c_, int i, int j, const int* n, const double* d, double r) {
  (void)j; (void)n; (void)i; (void)d;
  rdf_ctx* c = (rdf_ctx*)c_;
  const double norm = 1.0 / (sqrt(2.0 * M_PI) * c->w * 4.0 * M_PI);
  for (int k = 0; k < c->K; k++) {
    double rk = (k + 0.5) * c->D, t = (r - rk) / c->w;
    if (fabs(t) > 12.0) continue;
    c->g[k] += c->pref * exp(-0.5 * t * t) * norm / (rk * rk);
  }
}
/* gradient of sum_k gg_k g_k with respect to x (ordered pairs: d/dx_i of a
 * function of r_ij gets -u from (i,j) and -u again from (j,i)) */
static void rdf_bwd_cb(void* c_, int i, int j, const int* n, const double* d, double r) {
  (void)j; (void)n;
  rdf_ctx* c = (rdf_ctx*)c_;
  const double norm = 1.0 / (sqrt(2.0 * M_PI) * c->w * 4.0 * M_PI);
  double dG = 0;
  for (int k = 0; k < c->K; k++) {
    double rk = (k + 0.5) * c->D, t = (r - rk) / c->w;
    if (fabs(t) > 12.0) continue;
    dG += c->gg[k] * c->pref * exp(-0.5 * t * t) * norm / (rk * rk) * (-t / c->w);
  }
  for (int a = 0; a < 3; a++) c->gx[3 * i + a] -= 2.0 * dG * d[a] / r;
}
/* g [B,K] per system; if gg != NULL also gx [N,3] = d(sum_s sum_k gg[s,k] g[s,k])/dx */
void or_rdf(int B, const int64_t* offsets, const double* x, const double* cells, const uint8_t* pbc,
            double rmax, int K, int use_cells, double* g, const double* gg, double* gx) {
  if (gx) memset(gx, 0, sizeof(double) * 3 * offsets[B]);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < B; s++) {
    int64_t o = offsets[s]; int n = (int)(offsets[s + 1] - o);
    const double* h = cells + 9 * s;
    rdf_ctx c; c.K = K; c.D = rmax / K; c.w = c.D;
    c.pref = fabs(det3(h)) / ((double)n * (double)(n - 1));
    c.g = g + (size_t)K * s; c.gg = gg ? gg + (size_t)K * s : NULL; c.gx = gx ? gx + 3 * o : NULL;
    for (int k = 0; k < K; k++) c.g[k] = 0;
    double rcut = rmax + 4.0 * c.w;
    for_pairs(use_cells, n, x + 3 * o, h, pbc + 3 * s, rcut, rdf_cb, &c);
    if (gg) for_pairs(use_cells, n, x + 3 * o, h, pbc + 3 * s, rcut, rdf_bwd_cb, &c);
  }
}

/* ------------------------------------------------------------------------- */
/* Differentiable trajectory (Sec. 2): NVE velocity Verlet for T steps from   */
/* (x0, v0); frames every obs_every steps (t = obs_every, 2 obs_every, ...,  */
/* T); smeared RDF averaged over systems and frames; loss = (1/K) sum_k       */
/* (g_k - target_k)^2.  All systems share one potential (index 0 of pots).   */
/* Returns the loss; if gth != NULL also d loss / d params (3 values) by the  */
/* discrete adjoint of velocity Verlet, storing the whole trajectory (no      */
/* checkpointing: the oracle trades memory for plainness).                   */
/* Reverse of one step (c = dt/2m, u = x_{t+1}):                              */
/*   ubar = ax + c J(u)^T av;  vhbar = av + dt ubar;                          */
/*   ax <- ubar + c J(x_t)^T vhbar;  av <- vhbar;                             */
/*   gtheta += c Jtheta(u)^T av_old + c Jtheta(x_t)^T vhbar,                  */
/* with J = dF/dx applied through or_forces_backward.  Pinned by central      */
/* differences of the loss in the parameters.                                */
/* ------------------------------------------------------------------------- */
double or_traj_rdf_loss(int B, const int64_t* offsets, const double* x0, const double* v0, const double* mass,
                        const double* cells, const uint8_t* pbc, const or_pot* pot, int use_cells,
                        double dt, int T, int obs_every, double rmax, int K, const double* target,
                        double* g_out, double* gth) {
  int64_t N = offsets[B];
  int nfr = T / obs_every;
  size_t sz = sizeof(double) * 3 * N;
  int32_t* pos0 = (int32_t*)calloc(B, sizeof(int32_t));
  double* X = (double*)malloc(sz * (T + 1));
  double* Vv = (double*)malloc(sz * (T + 1));
  double* F = (double*)malloc(sz);
  double* E = (double*)malloc(sizeof(double) * B);
  double* g = (double*)calloc((size_t)K * B, sizeof(double));
  double* gacc = (double*)calloc(K, sizeof(double));
  memcpy(X, x0, sz); memcpy(Vv, v0, sz);
  or_forces(B, offsets, X, cells, pbc, pos0, pot, use_cells, E, F, NULL, NULL);
  for (int t = 0; t < T; t++) {
    double* x = X + 3 * N * t; double* v = Vv + 3 * N * t;
    double* xn = X + 3 * N * (t + 1); double* vn = Vv + 3 * N * (t + 1);
    for (int64_t i = 0; i < N; i++)
      for (int a = 0; a < 3; a++) {
        double vh = v[3 * i + a] + 0.5 * dt / mass[i] * F[3 * i + a];
        vn[3 * i + a] = vh;
        xn[3 * i + a] = x[3 * i + a] + dt * vh;
      }
    or_forces(B, offsets, xn, cells, pbc, pos0, pot, use_cells, E, F, NULL, NULL);
    for (int64_t i = 0; i < N; i++)
      for (int a = 0; a < 3; a++) vn[3 * i + a] += 0.5 * dt / mass[i] * F[3 * i + a];
    if ((t + 1) % obs_every == 0) {
      or_rdf(B, offsets, xn, cells, pbc, rmax, K, use_cells, g, NULL, NULL);
      for (int s = 0; s < B; s++)
        for (int k = 0; k < K; k++) gacc[k] += g[(size_t)K * s + k] / ((double)B * nfr);
    }
  }
  double loss = 0;
  for (int k = 0; k < K; k++) loss += (gacc[k] - target[k]) * (gacc[k] - target[k]) / K;
  if (g_out) memcpy(g_out, gacc, sizeof(double) * K);
  if (gth) {
    double* dg = (double*)malloc(sizeof(double) * K * B);
    for (int s = 0; s < B; s++)
      for (int k = 0; k < K; k++) dg[(size_t)K * s + k] = 2.0 * (gacc[k] - target[k]) / K / ((double)B * nfr);
    double* ax = (double*)calloc(3 * N, sizeof(double));
    double* av = (double*)calloc(3 * N, sizeof(double));
    double* ub = (double*)malloc(sz);
    double* vh = (double*)malloc(sz);
    double* gF = (double*)malloc(sz);
    double* tmp = (double*)malloc(sz);
    double gt[3];
    gth[0] = gth[1] = gth[2] = 0;
    for (int t = T - 1; t >= 0; t--) {
      double* x = X + 3 * N * t; double* u = X + 3 * N * (t + 1);
      if ((t + 1) % obs_every == 0) {   /* direct loss term at frame x_{t+1} */
        or_rdf(B, offsets, u, cells, pbc, rmax, K, use_cells, g, dg, tmp);
        for (int64_t q = 0; q < 3 * N; q++) ax[q] += tmp[q];
      }
      for (int64_t i = 0; i < N; i++) for (int a = 0; a < 3; a++) gF[3 * i + a] = 0.5 * dt / mass[i] * av[3 * i + a];
      or_forces_backward(B, offsets, u, cells, pbc, pos0, pot, 1, use_cells, gF, NULL, NULL, tmp, gt);
      for (int p = 0; p < 3; p++) gth[p] += gt[p];
      for (int64_t q = 0; q < 3 * N; q++) { ub[q] = ax[q] + tmp[q]; vh[q] = av[q] + dt * ub[q]; }
      for (int64_t i = 0; i < N; i++) for (int a = 0; a < 3; a++) gF[3 * i + a] = 0.5 * dt / mass[i] * vh[3 * i + a];
      or_forces_backward(B, offsets, x, cells, pbc, pos0, pot, 1, use_cells, gF, NULL, NULL, tmp, gt);
      for (int p = 0; p < 3; p++) gth[p] += gt[p];
      for (int64_t q = 0; q < 3 * N; q++) { ax[q] = ub[q] + tmp[q]; av[q] = vh[q]; }
    }
    free(dg); free(ax); free(av); free(ub); free(vh); free(gF); free(tmp);
  }
  free(pos0); free(X); free(Vv); free(F); free(E); free(g); free(gacc);
  return loss;
}

/* Number of OpenMP threads the oracle uses (for reporting). */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
