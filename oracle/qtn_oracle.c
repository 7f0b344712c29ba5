/*
 * Oracle for the QAOA single-amplitude tensor-network method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or table with the product.
 *
 * Everything is plain complex128 (C99 `double complex`), written for
 * readability, not speed.
 *
 * Quantity (definition): for a graph G = (V, E) on n qubits and p layers,
 *   a(x) = <x| U_B(beta_p) U_C(gamma_p) ... U_B(beta_1) U_C(gamma_1) H^n |0^n>,
 *   U_C(g) = prod_{(i,j) in E} exp(-i g Z_i Z_j),  U_B(b) = prod_i exp(-i b X_i).
 * Qubit i is bit i of a basis-state index (little endian).
 *
 * Three independent evaluations:
 *   oracle_statevector : the definition applied to a 2^n state vector.
 *   oracle_pathsum     : the definition expanded as a sum over computational
 *                        basis paths (every intermediate state), tiny n*p only.
 *   oracle_tn          : the paper's method.  The circuit becomes a tensor
 *                        network whose vertices are the input states, the
 *                        gates and the measurement, and whose edges are the
 *                        wire segments (Sec. II.A, Fig. 1; dimension 2 per
 *                        edge, the amplitude form).  Cut edges are fixed to
 *                        each of their values and the resulting subnetworks
 *                        are contracted one by one (Sec. III.A, Eq. 2); each
 *                        subnetwork is contracted pairwise (Eq. 1) along a
 *                        min-fill elimination order over its edges
 *                        (Sec. II.B), and the per-slice scalars are added
 *                        with a compensated (Kahan) sum, by worker threads
 *                        that each own a range of slices and a master that
 *                        adds their partial sums in order (Sec. III.A: one
 *                        scalar per subgraph goes back to the master).
 *
 * Parity pins (see tests): closed forms at gamma = 0, beta = 0, beta = pi/2;
 * dense matrix exponentials (scipy) for n <= 8; statevector <-> path sum <->
 * network on small n; sum |a|^2 = 1; sliced sum = unsliced contraction.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- gates -- */

/* exp(-i b X) = [[cos b, -i sin b], [-i sin b, cos b]]  (RX(2b)). */
static cplx rx_entry(double b, int row, int col) {
  return row == col ? cos(b) + 0.0 * I : -I * sin(b);
}

/* exp(-i g Z(x)Z) on |z1 z2>: eigenvalue of Z(x)Z is s1*s2, s = 1 - 2z. */
static cplx zz_phase(double g, int z1, int z2) {
  int s = (1 - 2 * z1) * (1 - 2 * z2);
  return cexp(-I * g * (double)s);
}

/* Edges are applied in lexicographic (i < j) order; they commute. */
static int cmp_edge(const void* a, const void* b) {
  const int32_t* x = (const int32_t*)a;
  const int32_t* y = (const int32_t*)b;
  if (x[0] != y[0]) return x[0] - y[0];
  return x[1] - y[1];
}

static int32_t* sorted_edges(const int32_t* edges, int m) {
  int32_t* e = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)m);
  for (int i = 0; i < m; ++i) {
    int a = edges[2 * i], b = edges[2 * i + 1];
    e[2 * i] = a < b ? a : b;
    e[2 * i + 1] = a < b ? b : a;
  }
  qsort(e, (size_t)m, 2 * sizeof(int32_t), cmp_edge);
  return e;
}

/* ------------------------------------------------------- state vector -- */

/* All 2^n amplitudes; out_re/out_im have 2^n entries.  Returns 0 on success. */
int oracle_statevector(int n, int p, const int32_t* edges, int m, const double* gamma,
                       const double* beta, double* out_re, double* out_im) {
  if (n < 1 || n > 28) return 1;
  size_t N = (size_t)1 << n;
  cplx* psi = (cplx*)malloc(sizeof(cplx) * N);
  if (!psi) return 2;
  double h = pow(2.0, -0.5 * n);
  for (size_t z = 0; z < N; ++z) psi[z] = h; /* H^n |0^n> */
  for (int l = 0; l < p; ++l) {
    for (size_t z = 0; z < N; ++z) { /* U_C: diagonal */
      cplx ph = 1.0;
      for (int e = 0; e < m; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        ph *= zz_phase(gamma[l], (int)((z >> a) & 1), (int)((z >> b) & 1));
      }
      psi[z] *= ph;
    }
    for (int q = 0; q < n; ++q) { /* U_B: one 2x2 per qubit */
      size_t bit = (size_t)1 << q;
      for (size_t z = 0; z < N; ++z) {
        if (z & bit) continue;
        cplx a0 = psi[z], a1 = psi[z | bit];
        psi[z] = rx_entry(beta[l], 0, 0) * a0 + rx_entry(beta[l], 0, 1) * a1;
        psi[z | bit] = rx_entry(beta[l], 1, 0) * a0 + rx_entry(beta[l], 1, 1) * a1;
      }
    }
  }
  for (size_t z = 0; z < N; ++z) {
    out_re[z] = creal(psi[z]);
    out_im[z] = cimag(psi[z]);
  }
  free(psi);
  return 0;
}

/* ----------------------------------------------------------- path sum -- */

/* a(x) = sum over z^(1), ..., z^(p) of
 *   2^{-n/2} prod_l [ exp(-i gamma_l sum_E s_i s_j (z^(l))) prod_i <z_i^(l+1)| e^{-i beta_l X} |z_i^(l)> ],
 * with z^(p+1) = x.  Exponential in n*p: only for n*p <= 24. */
int oracle_pathsum(int n, int p, const int32_t* edges, int m, const double* gamma,
                   const double* beta, uint64_t x, double out[2]) {
  if (n * p > 24 || n > 62) return 1;
  uint64_t per = (uint64_t)1 << n;
  uint64_t total = (uint64_t)1 << (n * p);
  cplx sum = 0, comp = 0; /* compensated (Kahan) sum over 2^(n p) paths */
  for (uint64_t path = 0; path < total; ++path) {
    cplx term = 1;
    for (int l = 0; l < p; ++l) {
      uint64_t z = (path >> (n * l)) & (per - 1);
      uint64_t znext = (l + 1 < p) ? ((path >> (n * (l + 1))) & (per - 1)) : x;
      double ising = 0;
      for (int e = 0; e < m; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        ising += (double)((1 - 2 * (int)((z >> a) & 1)) * (1 - 2 * (int)((z >> b) & 1)));
      }
      term *= cexp(-I * gamma[l] * ising);
      for (int q = 0; q < n; ++q)
        term *= rx_entry(beta[l], (int)((znext >> q) & 1), (int)((z >> q) & 1));
    }
    cplx y = term - comp;
    cplx t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  sum *= pow(2.0, -0.5 * n);
  out[0] = creal(sum);
  out[1] = cimag(sum);
  return 0;
}

/* ------------------------------------------------------ tensor network -- */

/* A dense tensor: `rank` edge labels; entry for label values (v_0..v_{r-1})
 * is data[sum_j v_j << j]. */
typedef struct {
  int rank;
  int* labels;
  cplx* data;
} Tensor;

/* The circuit as a network of vertices (tensors) joined by wire segments
 * (edge labels).  On each qubit the vertices are, in time order:
 *   input |0>, H, [ZZ gates of layer l ..., RX(2 beta_l)] for l = 1..p, <x_q|.
 * A wire segment is labelled by its id; seg_zz_in[q][t] is the label of the
 * segment that enters the t-th ZZ gate acting on qubit q. */
typedef struct {
  int n_tensors;
  Tensor* t;
  int n_labels;
  int* zz_in_label; /* [q * max_zz + t] */
  int* zz_count;    /* ZZ gates per qubit */
  int max_zz;
} Circuit;

static Tensor tensor_new(int rank) {
  Tensor T;
  T.rank = rank;
  T.labels = (int*)malloc(sizeof(int) * (rank > 0 ? rank : 1));
  T.data = (cplx*)calloc((size_t)1 << rank, sizeof(cplx));
  return T;
}

static void tensor_free(Tensor* T) {
  free(T->labels);
  free(T->data);
  T->labels = NULL;
  T->data = NULL;
}

static void circuit_free(Circuit* c) {
  for (int i = 0; i < c->n_tensors; ++i) tensor_free(&c->t[i]);
  free(c->t);
  free(c->zz_in_label);
  free(c->zz_count);
}

static void circuit_build(int n, int p, const int32_t* edges_in, int m, const double* gamma,
                          const double* beta, uint64_t x_lo, const uint8_t* xbits, Circuit* c) {
  int32_t* edges = sorted_edges(edges_in, m);
  int cap = 3 * n + 2 * n * p + m * p + 4;
  c->t = (Tensor*)malloc(sizeof(Tensor) * (size_t)cap);
  c->n_tensors = 0;
  c->n_labels = 0;
  c->zz_count = (int*)calloc((size_t)n, sizeof(int));
  for (int e = 0; e < m; ++e) {
    c->zz_count[edges[2 * e]] += p;
    c->zz_count[edges[2 * e + 1]] += p;
  }
  c->max_zz = 1;
  for (int q = 0; q < n; ++q)
    if (c->zz_count[q] > c->max_zz) c->max_zz = c->zz_count[q];
  c->zz_in_label = (int*)malloc(sizeof(int) * (size_t)n * (size_t)c->max_zz);
  int* open = (int*)malloc(sizeof(int) * (size_t)n); /* label of the open wire end */
  int* seen = (int*)calloc((size_t)n, sizeof(int));
  const double h = 1.0 / sqrt(2.0);
  for (int q = 0; q < n; ++q) {
    Tensor in = tensor_new(1); /* |0> */
    in.labels[0] = c->n_labels++;
    in.data[0] = 1.0;
    c->t[c->n_tensors++] = in;
    Tensor H = tensor_new(2); /* H[out, in] */
    H.labels[0] = c->n_labels++;
    H.labels[1] = in.labels[0];
    H.data[0] = h;  /* out 0, in 0 */
    H.data[1] = h;  /* out 1, in 0 */
    H.data[2] = h;  /* out 0, in 1 */
    H.data[3] = -h; /* out 1, in 1 */
    c->t[c->n_tensors++] = H;
    open[q] = H.labels[0];
  }
  for (int l = 0; l < p; ++l) {
    for (int e = 0; e < m; ++e) {
      int a = edges[2 * e], b = edges[2 * e + 1];
      /* ZZ[out_a, out_b, in_a, in_b] = delta(out_a,in_a) delta(out_b,in_b) phase */
      Tensor Z = tensor_new(4);
      Z.labels[0] = c->n_labels++;
      Z.labels[1] = c->n_labels++;
      Z.labels[2] = open[a];
      Z.labels[3] = open[b];
      c->zz_in_label[a * c->max_zz + seen[a]++] = open[a];
      c->zz_in_label[b * c->max_zz + seen[b]++] = open[b];
      for (int za = 0; za < 2; ++za)
        for (int zb = 0; zb < 2; ++zb)
          Z.data[za | (zb << 1) | (za << 2) | (zb << 3)] = zz_phase(gamma[l], za, zb);
      c->t[c->n_tensors++] = Z;
      open[a] = Z.labels[0];
      open[b] = Z.labels[1];
    }
    for (int q = 0; q < n; ++q) {
      Tensor R = tensor_new(2); /* R[out, in] */
      R.labels[0] = c->n_labels++;
      R.labels[1] = open[q];
      for (int o = 0; o < 2; ++o)
        for (int i2 = 0; i2 < 2; ++i2) R.data[o | (i2 << 1)] = rx_entry(beta[l], o, i2);
      c->t[c->n_tensors++] = R;
      open[q] = R.labels[0];
    }
  }
  for (int q = 0; q < n; ++q) {
    int bit = xbits ? xbits[q] : (int)((x_lo >> q) & 1);
    Tensor O = tensor_new(1); /* <x_q| */
    O.labels[0] = open[q];
    O.data[bit] = 1.0;
    O.data[1 - bit] = 0.0;
    c->t[c->n_tensors++] = O;
  }
  free(open);
  free(seen);
  free(edges);
}

/* Sub-block of T with edge `label` fixed to `value` (the edge is removed). */
static Tensor tensor_fix(const Tensor* T, int label, int value) {
  int pos = -1;
  for (int j = 0; j < T->rank; ++j)
    if (T->labels[j] == label) pos = j;
  Tensor R = tensor_new(T->rank - 1);
  for (int j = 0, r = 0; j < T->rank; ++j)
    if (j != pos) R.labels[r++] = T->labels[j];
  size_t NR = (size_t)1 << R.rank;
  for (size_t o = 0; o < NR; ++o) {
    size_t low = o & (((size_t)1 << pos) - 1);
    size_t high = o >> pos;
    size_t src = low | ((size_t)value << pos) | (high << (pos + 1));
    R.data[o] = T->data[src];
  }
  return R;
}

static int has_label(const Tensor* T, int label) {
  for (int j = 0; j < T->rank; ++j)
    if (T->labels[j] == label) return 1;
  return 0;
}

/* Eq. (1): g = sum over shared edges of e * f; the result keeps the edges of
 * e that f lacks, then the edges of f that e lacks.  Instrumented with the
 * number of complex multiply-adds it performs. */
static Tensor contract_pair(const Tensor* e, const Tensor* f, double* macs) {
  int shared = 0;
  for (int j = 0; j < e->rank; ++j) shared += has_label(f, e->labels[j]);
  int rank = e->rank + f->rank - 2 * shared;
  Tensor g = tensor_new(rank);
  int r = 0;
  for (int j = 0; j < e->rank; ++j)
    if (!has_label(f, e->labels[j])) g.labels[r++] = e->labels[j];
  for (int j = 0; j < f->rank; ++j)
    if (!has_label(e, f->labels[j])) g.labels[r++] = f->labels[j];
  /* All edges of the pair: g's edges, then the shared ones. */
  int nall = rank + shared;
  int* all = (int*)malloc(sizeof(int) * (nall > 0 ? nall : 1));
  for (int j = 0; j < rank; ++j) all[j] = g.labels[j];
  for (int j = 0, s = rank; j < e->rank; ++j)
    if (has_label(f, e->labels[j])) all[s++] = e->labels[j];
  /* Position in `all` of each edge of e and f. */
  int* pe = (int*)malloc(sizeof(int) * (e->rank > 0 ? e->rank : 1));
  int* pf = (int*)malloc(sizeof(int) * (f->rank > 0 ? f->rank : 1));
  for (int j = 0; j < e->rank; ++j)
    for (int a = 0; a < nall; ++a)
      if (all[a] == e->labels[j]) pe[j] = a;
  for (int j = 0; j < f->rank; ++j)
    for (int a = 0; a < nall; ++a)
      if (all[a] == f->labels[j]) pf[j] = a;
  size_t NA = (size_t)1 << nall;
  size_t NG = (size_t)1 << rank;
  for (size_t v = 0; v < NA; ++v) { /* one assignment of every edge */
    size_t ie = 0, jf = 0;
    for (int j = 0; j < e->rank; ++j) ie |= ((v >> pe[j]) & 1) << j;
    for (int j = 0; j < f->rank; ++j) jf |= ((v >> pf[j]) & 1) << j;
    g.data[v & (NG - 1)] += e->data[ie] * f->data[jf];
  }
  *macs += (double)NA;
  free(all);
  free(pe);
  free(pf);
  return g;
}

/* Min-fill elimination order over the edges of a network (Sec. II.B):
 * repeatedly eliminate the edge whose two endpoint tensors, once merged,
 * create the fewest new co-occurrences of edges; ties by the merged tensor's
 * size, then by label.  Works on a copy of the label sets. */
static int* minfill_order(int nt, const Tensor* ts, int n_labels, int* n_order) {
  int** sets = (int**)malloc(sizeof(int*) * (size_t)nt * 2);
  int* sz = (int*)calloc((size_t)nt * 2, sizeof(int));
  char* alive_t = (char*)calloc((size_t)nt * 2, 1);
  for (int i = 0; i < nt; ++i) {
    sets[i] = (int*)malloc(sizeof(int) * (size_t)n_labels);
    sz[i] = ts[i].rank;
    memcpy(sets[i], ts[i].labels, sizeof(int) * (size_t)ts[i].rank);
    alive_t[i] = 1;
  }
  int count = nt;
  char* alive_l = (char*)calloc((size_t)n_labels, 1);
  int nalive = 0;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < sz[i]; ++j)
      if (!alive_l[sets[i][j]]) {
        alive_l[sets[i][j]] = 1;
        nalive++;
      }
  /* adj[u*n_labels+v]: u and v are in a common live tensor */
  char* adj = (char*)calloc((size_t)n_labels * (size_t)n_labels, 1);
  for (int i = 0; i < nt; ++i)
    for (int a = 0; a < sz[i]; ++a)
      for (int b = 0; b < sz[i]; ++b) adj[(size_t)sets[i][a] * n_labels + sets[i][b]] = 1;
  int* order = (int*)malloc(sizeof(int) * (size_t)(n_labels > 0 ? n_labels : 1));
  int no = 0;
  int* holder = (int*)malloc(sizeof(int) * 2 * (size_t)n_labels);
  while (nalive > 0) {
    int best = -1, best_t1 = -1, best_t2 = -1;
    long best_fill = -1, best_size = 0;
    /* the two live tensors that hold each live edge */
    for (int u = 0; u < 2 * n_labels; ++u) holder[u] = -1;
    for (int i = 0; i < count; ++i) {
      if (!alive_t[i]) continue;
      for (int j = 0; j < sz[i]; ++j) {
        int u = sets[i][j];
        if (holder[2 * u] < 0) holder[2 * u] = i;
        else holder[2 * u + 1] = i;
      }
    }
    for (int u = 0; u < n_labels; ++u) {
      if (!alive_l[u]) continue;
      int t1 = holder[2 * u], t2 = holder[2 * u + 1];
      long fill = 0, size = 0;
      for (int a = 0; a < sz[t1]; ++a) {
        int in2 = 0;
        for (int b = 0; b < sz[t2]; ++b) in2 |= sets[t2][b] == sets[t1][a];
        if (in2) continue;
        for (int b = 0; b < sz[t2]; ++b) {
          int in1 = 0;
          for (int c2 = 0; c2 < sz[t1]; ++c2) in1 |= sets[t1][c2] == sets[t2][b];
          if (in1) continue;
          if (!adj[(size_t)sets[t1][a] * n_labels + sets[t2][b]]) fill++;
        }
      }
      size = sz[t1] + sz[t2];
      if (best < 0 || fill < best_fill || (fill == best_fill && size < best_size)) {
        best = u;
        best_fill = fill;
        best_size = size;
        best_t1 = t1;
        best_t2 = t2;
      }
    }
    order[no++] = best;
    /* merge best_t1, best_t2: symmetric difference; shared labels die */
    int nt3 = count++;
    sets[nt3] = (int*)malloc(sizeof(int) * (size_t)n_labels);
    sz[nt3] = 0;
    alive_t[nt3] = 1;
    for (int pass = 0; pass < 2; ++pass) {
      int ta = pass == 0 ? best_t1 : best_t2, tb = pass == 0 ? best_t2 : best_t1;
      for (int a = 0; a < sz[ta]; ++a) {
        int shared = 0;
        for (int b = 0; b < sz[tb]; ++b) shared |= sets[tb][b] == sets[ta][a];
        if (shared) {
          if (alive_l[sets[ta][a]]) {
            alive_l[sets[ta][a]] = 0;
            nalive--;
          }
        } else {
          sets[nt3][sz[nt3]++] = sets[ta][a];
        }
      }
    }
    for (int a = 0; a < sz[nt3]; ++a)
      for (int b = 0; b < sz[nt3]; ++b) adj[(size_t)sets[nt3][a] * n_labels + sets[nt3][b]] = 1;
    alive_t[best_t1] = alive_t[best_t2] = 0;
  }
  for (int i = 0; i < count; ++i) free(sets[i]);
  free(sets);
  free(sz);
  free(alive_t);
  free(alive_l);
  free(adj);
  free(holder);
  *n_order = no;
  return order;
}

/* Contract a closed network (every edge on exactly two tensors) to a scalar
 * along `order`: for each edge, merge the two tensors holding it (Eq. 1);
 * then multiply the remaining scalars.  Consumes `ts`. */
static cplx contract_network(int nt, Tensor* ts, const int* order, int n_order, double* macs) {
  Tensor* live = (Tensor*)malloc(sizeof(Tensor) * (size_t)nt);
  char* alive = (char*)malloc((size_t)nt);
  for (int i = 0; i < nt; ++i) {
    live[i] = ts[i];
    alive[i] = 1;
  }
  for (int s = 0; s < n_order; ++s) {
    int u = order[s], t1 = -1, t2 = -1;
    for (int i = 0; i < nt; ++i)
      if (alive[i] && has_label(&live[i], u)) {
        if (t1 < 0) t1 = i;
        else t2 = i;
      }
    if (t1 < 0 || t2 < 0) continue; /* already summed with an earlier edge */
    Tensor g = contract_pair(&live[t1], &live[t2], macs);
    tensor_free(&live[t1]);
    tensor_free(&live[t2]);
    alive[t2] = 0;
    live[t1] = g;
  }
  cplx r = 1;
  for (int i = 0; i < nt; ++i)
    if (alive[i]) {
      r *= live[i].data[0]; /* rank 0 by now */
      *macs += 1;
      tensor_free(&live[i]);
    }
  free(live);
  free(alive);
  return r;
}

typedef struct {
  const Circuit* c;
  const int* cut_labels;
  int k;
  const int* order;
  int n_order;
  uint64_t lo, hi;       /* slice range [lo, hi) */
  double* per_slice;     /* optional: (re, im) per slice, indexed s - base */
  uint64_t base;
  cplx sum, comp;        /* Kahan partial sum of the range */
  double macs;
} Work;

static void kahan_add(cplx* sum, cplx* comp, cplx v) {
  cplx y = v - *comp;
  cplx t = *sum + y;
  *comp = (t - *sum) - y;
  *sum = t;
}

/* Build the sliced network of slice s (cut j fixed to bit j of s). */
static Tensor* sliced_network(const Circuit* c, const int* cut_labels, int k, uint64_t s) {
  Tensor* ts = (Tensor*)malloc(sizeof(Tensor) * (size_t)c->n_tensors);
  for (int i = 0; i < c->n_tensors; ++i) {
    Tensor cur = tensor_new(c->t[i].rank);
    memcpy(cur.labels, c->t[i].labels, sizeof(int) * (size_t)cur.rank);
    memcpy(cur.data, c->t[i].data, sizeof(cplx) * ((size_t)1 << cur.rank));
    for (int j = 0; j < k; ++j)
      if (has_label(&cur, cut_labels[j])) {
        Tensor f = tensor_fix(&cur, cut_labels[j], (int)((s >> j) & 1));
        tensor_free(&cur);
        cur = f;
      }
    ts[i] = cur;
  }
  return ts;
}

static void* worker(void* arg) {
  Work* w = (Work*)arg;
  w->sum = 0;
  w->comp = 0;
  w->macs = 0;
  for (uint64_t s = w->lo; s < w->hi; ++s) {
    Tensor* ts = sliced_network(w->c, w->cut_labels, w->k, s);
    cplx v = contract_network(w->c->n_tensors, ts, w->order, w->n_order, &w->macs);
    free(ts);
    if (w->per_slice) {
      w->per_slice[2 * (s - w->base)] = creal(v);
      w->per_slice[2 * (s - w->base) + 1] = cimag(v);
    }
    kahan_add(&w->sum, &w->comp, v);
  }
  return NULL;
}

/*
 * The paper's method on the host.
 *   x            : n bytes, x[q] = measured bit of qubit q.
 *   cut_qubit[j], cut_pos[j] (j < k): cut the wire segment that enters the
 *                  (cut_pos[j] + 1)-th ZZ gate (0-based count cut_pos[j]+1)
 *                  acting on qubit cut_qubit[j]; requires
 *                  0 <= cut_pos[j] < (ZZ gates on that qubit) - 1.
 *   slices [slice_lo, slice_hi) of the 2^k are contracted (slice s fixes cut
 *   j to bit j of s) and summed; pass 0 and 2^k for the full amplitude.
 *   threads      : worker threads (>= 1).
 *   out[2]       : the (Kahan) sum over the range.
 *   per_slice    : optional, 2 * (slice_hi - slice_lo) doubles.
 *   macs_out     : optional, complex multiply-adds performed.
 *   width_out    : optional, max rank of any tensor merged by the order
 *                  (max |A u B| over pairwise contractions).
 * Returns 0 on success.
 */
int oracle_tn(int n, int p, const int32_t* edges, int m, const double* gamma, const double* beta,
              const uint8_t* x, const int32_t* cut_qubit, const int32_t* cut_pos, int k,
              uint64_t slice_lo, uint64_t slice_hi, int threads, double out[2], double* per_slice,
              double* macs_out, int* width_out) {
  if (n < 1 || p < 1 || m < 1 || k < 0 || k > 62 || threads < 1) return 1;
  if (slice_hi > ((uint64_t)1 << k) || slice_lo > slice_hi) return 1;
  Circuit c;
  circuit_build(n, p, edges, m, gamma, beta, 0, x, &c);
  int* cut_labels = (int*)malloc(sizeof(int) * (size_t)(k > 0 ? k : 1));
  for (int j = 0; j < k; ++j) {
    int q = cut_qubit[j], t = cut_pos[j];
    if (q < 0 || q >= n || t < 0 || t + 1 >= c.zz_count[q]) {
      free(cut_labels);
      circuit_free(&c);
      return 2;
    }
    cut_labels[j] = c.zz_in_label[q * c.max_zz + t + 1];
    for (int i = 0; i < j; ++i)
      if (cut_labels[i] == cut_labels[j]) {
        free(cut_labels);
        circuit_free(&c);
        return 3;
      }
  }
  /* The order is planned once, on slice 0's network (all slices share it). */
  Tensor* s0 = sliced_network(&c, cut_labels, k, 0);
  int n_order = 0;
  int* order = minfill_order(c.n_tensors, s0, c.n_labels, &n_order);
  if (width_out) {
    /* replay the order on label sets to get the largest pairwise union */
    double dummy = 0;
    int width = 0;
    Tensor* ts = sliced_network(&c, cut_labels, k, 0);
    char* alive = (char*)malloc((size_t)c.n_tensors);
    memset(alive, 1, (size_t)c.n_tensors);
    for (int s = 0; s < n_order; ++s) {
      int u = order[s], t1 = -1, t2 = -1;
      for (int i = 0; i < c.n_tensors; ++i)
        if (alive[i] && has_label(&ts[i], u)) {
          if (t1 < 0) t1 = i;
          else t2 = i;
        }
      if (t1 < 0 || t2 < 0) continue;
      int shared = 0;
      for (int j = 0; j < ts[t1].rank; ++j) shared += has_label(&ts[t2], ts[t1].labels[j]);
      int uni = ts[t1].rank + ts[t2].rank - shared;
      if (uni > width) width = uni;
      Tensor g = contract_pair(&ts[t1], &ts[t2], &dummy);
      tensor_free(&ts[t1]);
      tensor_free(&ts[t2]);
      alive[t2] = 0;
      ts[t1] = g;
    }
    for (int i = 0; i < c.n_tensors; ++i)
      if (alive[i]) tensor_free(&ts[i]);
    free(ts);
    free(alive);
    *width_out = width;
  }
  for (int i = 0; i < c.n_tensors; ++i) tensor_free(&s0[i]);
  free(s0);

  uint64_t total = slice_hi - slice_lo;
  if ((uint64_t)threads > total && total > 0) threads = (int)total;
  if (total == 0) threads = 1;
  Work* w = (Work*)calloc((size_t)threads, sizeof(Work));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  for (int i = 0; i < threads; ++i) {
    w[i].c = &c;
    w[i].cut_labels = cut_labels;
    w[i].k = k;
    w[i].order = order;
    w[i].n_order = n_order;
    w[i].lo = slice_lo + total * (uint64_t)i / (uint64_t)threads;
    w[i].hi = slice_lo + total * (uint64_t)(i + 1) / (uint64_t)threads;
    w[i].per_slice = per_slice;
    w[i].base = slice_lo;
    if (threads > 1) pthread_create(&th[i], NULL, worker, &w[i]);
  }
  if (threads == 1) worker(&w[0]);
  cplx sum = 0, comp = 0;
  double macs = 0;
  for (int i = 0; i < threads; ++i) { /* master: fixed order */
    if (threads > 1) pthread_join(th[i], NULL);
    kahan_add(&sum, &comp, w[i].sum);
    macs += w[i].macs;
  }
  out[0] = creal(sum);
  out[1] = cimag(sum);
  if (macs_out) *macs_out = macs;
  free(w);
  free(th);
  free(order);
  free(cut_labels);
  circuit_free(&c);
  return 0;
}

/* Number of ZZ gates acting on each qubit (p * degree); for naming cuts. */
int oracle_zz_per_qubit(int n, int p, const int32_t* edges, int m, int32_t* out) {
  for (int q = 0; q < n; ++q) out[q] = 0;
  for (int e = 0; e < m; ++e) {
    out[edges[2 * e]] += p;
    out[edges[2 * e + 1]] += p;
  }
  return 0;
}

/* ------------------------------------------------ the oracle's own cuts -- */

/* Largest merged rank |A u B| of the min-fill order (Sec. II.B) of the
 * network with `cut_labels` removed, replayed on label sets only.  If
 * `counts` is given, every label of every merge of that largest rank gets
 * one count there. */
static int order_width(const Circuit* c, const int* cut_labels, int k, int* counts) {
  Tensor* ts = sliced_network(c, cut_labels, k, 0);
  int n_order = 0;
  int* order = minfill_order(c->n_tensors, ts, c->n_labels, &n_order);
  int nt = c->n_tensors;
  int** sets = (int**)malloc(sizeof(int*) * (size_t)nt);
  int* sz = (int*)malloc(sizeof(int) * (size_t)nt);
  char* alive = (char*)malloc((size_t)nt);
  for (int i = 0; i < nt; ++i) {
    sets[i] = (int*)malloc(sizeof(int) * (size_t)c->n_labels);
    sz[i] = ts[i].rank;
    memcpy(sets[i], ts[i].labels, sizeof(int) * (size_t)ts[i].rank);
    alive[i] = 1;
    tensor_free(&ts[i]);
  }
  free(ts);
  int* uni = (int*)malloc(sizeof(int) * (size_t)c->n_labels);
  int width = 0;
  for (int pass = 0; pass < (counts ? 2 : 1); ++pass) {
    /* pass 0 finds the width, pass 1 counts the labels of the widest merges */
    int** ws = (int**)malloc(sizeof(int*) * (size_t)nt);
    int* wz = (int*)malloc(sizeof(int) * (size_t)nt);
    char* wa = (char*)malloc((size_t)nt);
    for (int i = 0; i < nt; ++i) {
      ws[i] = (int*)malloc(sizeof(int) * (size_t)c->n_labels);
      memcpy(ws[i], sets[i], sizeof(int) * (size_t)sz[i]);
      wz[i] = sz[i];
      wa[i] = alive[i];
    }
    for (int s = 0; s < n_order; ++s) {
      int u = order[s], t1 = -1, t2 = -1;
      for (int i = 0; i < nt; ++i) {
        if (!wa[i]) continue;
        for (int j = 0; j < wz[i]; ++j)
          if (ws[i][j] == u) {
            if (t1 < 0) t1 = i;
            else t2 = i;
          }
      }
      if (t1 < 0 || t2 < 0) continue;
      int nu = 0;
      for (int j = 0; j < wz[t1]; ++j) uni[nu++] = ws[t1][j];
      for (int j = 0; j < wz[t2]; ++j) {
        int dup = 0;
        for (int a = 0; a < wz[t1]; ++a) dup |= ws[t1][a] == ws[t2][j];
        if (!dup) uni[nu++] = ws[t2][j];
      }
      if (pass == 0 && nu > width) width = nu;
      if (pass == 1 && nu == width)
        for (int j = 0; j < nu; ++j) counts[uni[j]]++;
      /* merged tensor: labels of the union held by only one of the two */
      int nr = 0;
      for (int j = 0; j < nu; ++j) {
        int in1 = 0, in2 = 0;
        for (int a = 0; a < wz[t1]; ++a) in1 |= ws[t1][a] == uni[j];
        for (int a = 0; a < wz[t2]; ++a) in2 |= ws[t2][a] == uni[j];
        if (!(in1 && in2)) ws[t1][nr++] = uni[j];
      }
      wz[t1] = nr;
      wa[t2] = 0;
    }
    for (int i = 0; i < nt; ++i) free(ws[i]);
    free(ws);
    free(wz);
    free(wa);
  }
  for (int i = 0; i < nt; ++i) free(sets[i]);
  free(sets);
  free(sz);
  free(alive);
  free(uni);
  free(order);
  return width;
}

/*
 * The oracle's own cut set of k wire segments, chosen without the product's
 * planner (Sec. III.A: cutting edges lowers the width of the subnetworks).
 * k times: plan the min-fill order of the network with the cuts chosen so
 * far removed, find its largest merged rank, and cut the candidate segment
 * that occurs in the most merges of that rank (ties: the lowest label; if
 * none occurs there, the lowest unused candidate).  Candidates are the
 * segments oracle_tn can name: those entering a ZZ gate other than the first
 * one on their qubit.  Writes (cut_qubit[j], cut_pos[j]) in oracle_tn's
 * naming and, if width_out is given, the width left by all k cuts.
 * Returns 0 on success, 1 for bad arguments or too few candidates.
 */
int oracle_choose_cuts(int n, int p, const int32_t* edges, int m, int k, int32_t* cut_qubit, int32_t* cut_pos,
                       int* width_out) {
  if (n < 1 || p < 1 || m < 1 || k < 0) return 1;
  double* zero = (double*)calloc((size_t)p, sizeof(double));
  Circuit c;
  circuit_build(n, p, edges, m, zero, zero, 0, NULL, &c);
  free(zero);
  int* cand_q = (int*)malloc(sizeof(int) * (size_t)c.n_labels);
  int* cand_t = (int*)malloc(sizeof(int) * (size_t)c.n_labels);
  for (int l = 0; l < c.n_labels; ++l) cand_q[l] = -1;
  int n_cand = 0;
  for (int q = 0; q < n; ++q)
    for (int t = 1; t < c.zz_count[q]; ++t) {
      int l = c.zz_in_label[q * c.max_zz + t];
      cand_q[l] = q;
      cand_t[l] = t - 1;
      n_cand++;
    }
  if (k > n_cand) {
    free(cand_q);
    free(cand_t);
    circuit_free(&c);
    return 1;
  }
  int* cut_labels = (int*)malloc(sizeof(int) * (size_t)(k > 0 ? k : 1));
  int* counts = (int*)malloc(sizeof(int) * (size_t)c.n_labels);
  for (int j = 0; j < k; ++j) {
    for (int l = 0; l < c.n_labels; ++l) counts[l] = 0;
    order_width(&c, cut_labels, j, counts);
    int best = -1;
    for (int l = 0; l < c.n_labels; ++l) {
      if (cand_q[l] < 0) continue;
      int used = 0;
      for (int i = 0; i < j; ++i) used |= cut_labels[i] == l;
      if (used) continue;
      if (best < 0 || counts[l] > counts[best]) best = l;
    }
    cut_labels[j] = best;
    cut_qubit[j] = cand_q[best];
    cut_pos[j] = cand_t[best];
  }
  if (width_out) *width_out = order_width(&c, cut_labels, k, NULL);
  free(counts);
  free(cut_labels);
  free(cand_q);
  free(cand_t);
  circuit_free(&c);
  return 0;
}
