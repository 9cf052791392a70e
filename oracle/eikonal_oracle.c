/*
 * eikonal_oracle.c — plain FP64 CPU reference of the first-arrival traveltime
 * solver.  TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg); the
 * library never uses it and it shares no code with the CUDA solver.
 *
 * The tomography stage of "A workflow for seismic imaging with quantified
 * uncertainty" (arXiv 2001.06444, §2.1 Eq. 1 and §3) links velocity to first
 * arrival traveltimes through the eikonal equation |grad T| = s = 1/v, solved
 * by fast marching (the FaATSO code).  Discretisation (the paper does not give
 * one; this is the standard first-order upwind scheme of fast marching):
 * nodes (i, j) on an nz x nx grid with spacings dz, dx; with a the smaller
 * vertical neighbour time and b the smaller horizontal one (infinite outside
 * the grid or when unknown), T solves
 *     ((T - a)^+ / dz)^2 + ((T - b)^+ / dx)^2 = s^2,
 * i.e. with u1 = min(a, b) (spacing h1) and u2 the other (h2): T = u1 + s h1
 * if that is <= u2, else the larger root of the two-term quadratic
 *     T = (w1 u1 + w2 u2 + sqrt((w1 + w2) s^2 - w1 w2 (u1 - u2)^2)) / (w1 + w2),
 * w = 1/h^2.  Source nodes hold T = 0.  Fast marching (Sethian 1996) accepts
 * nodes in increasing T from a binary heap and updates their neighbours from
 * the accepted ones.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The upwind update of one node from its smaller neighbours a (vertical)
 * and b (horizontal); INFINITY when both are unknown. */
double oracle_eikonal_update(double a, double b, double s, double dz, double dx) {
  double u1 = a, h1 = dz, u2 = b, h2 = dx;
  if (u1 > u2) {
    u1 = b;
    h1 = dx;
    u2 = a;
    h2 = dz;
  }
  if (isinf(u1)) return INFINITY;
  const double t1 = u1 + s * h1;
  if (t1 <= u2) return t1;
  const double w1 = 1.0 / (h1 * h1), w2 = 1.0 / (h2 * h2), d = u1 - u2;
  return (w1 * u1 + w2 * u2 + sqrt((w1 + w2) * s * s - w1 * w2 * d * d)) / (w1 + w2);
}

typedef struct {
  double t;
  int64_t k;
} item;

typedef struct {
  item *a;
  int64_t n, cap;
} heap;

static int heap_push(heap *h, double t, int64_t k) {
  if (h->n == h->cap) {
    const int64_t cap = h->cap ? 2 * h->cap : 1024;
    item *p = (item *)realloc(h->a, (size_t)cap * sizeof(item));
    if (!p) return -1;
    h->a = p;
    h->cap = cap;
  }
  int64_t i = h->n++;
  while (i > 0) {
    const int64_t up = (i - 1) / 2;
    if (h->a[up].t <= t) break;
    h->a[i] = h->a[up];
    i = up;
  }
  h->a[i].t = t;
  h->a[i].k = k;
  return 0;
}

static item heap_pop(heap *h) {
  const item top = h->a[0], last = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= h->n) break;
    if (c + 1 < h->n && h->a[c + 1].t < h->a[c].t) c++;
    if (h->a[c].t >= last.t) break;
    h->a[i] = h->a[c];
    i = c;
  }
  if (h->n > 0) h->a[i] = last;
  return top;
}

/* Traveltimes T [nz][nx] from the source nodes (src_iz[k], src_ix[k]),
 * k < nsrc, all at T = 0, for slowness s [nz][nx].  Returns 0, or -1 on bad
 * arguments or no memory. */
int oracle_eikonal(int nz, int nx, double dz, double dx, const double *s, int nsrc,
                   const int *src_iz, const int *src_ix, double *T) {
  if (nz < 1 || nx < 1 || !(dz > 0) || !(dx > 0) || nsrc < 1) return -1;
  const int64_t n = (int64_t)nz * nx;
  unsigned char *known = (unsigned char *)calloc((size_t)n, 1);
  heap h = {0, 0, 0};
  if (!known) return -1;
  for (int64_t k = 0; k < n; ++k) T[k] = INFINITY;
  int rc = 0;
  for (int k = 0; k < nsrc; ++k) {
    if (src_iz[k] < 0 || src_iz[k] >= nz || src_ix[k] < 0 || src_ix[k] >= nx) {
      rc = -1;
      break;
    }
    const int64_t id = (int64_t)src_iz[k] * nx + src_ix[k];
    T[id] = 0.0;
    if (heap_push(&h, 0.0, id)) rc = -1;
  }
  while (!rc && h.n > 0) {
    const item it = heap_pop(&h);
    if (known[it.k] || it.t > T[it.k]) continue; /* stale entry */
    known[it.k] = 1;
    const int i = (int)(it.k / nx), j = (int)(it.k % nx);
    const int ni[4] = {i - 1, i + 1, i, i}, nj[4] = {j, j, j - 1, j + 1};
    for (int q = 0; q < 4; ++q) {
      const int y = ni[q], x = nj[q];
      if (y < 0 || y >= nz || x < 0 || x >= nx) continue;
      const int64_t id = (int64_t)y * nx + x;
      if (known[id]) continue;
      double a = INFINITY, b = INFINITY;
      if (y > 0 && known[id - nx]) a = T[id - nx];
      if (y < nz - 1 && known[id + nx] && T[id + nx] < a) a = T[id + nx];
      if (x > 0 && known[id - 1]) b = T[id - 1];
      if (x < nx - 1 && known[id + 1] && T[id + 1] < b) b = T[id + 1];
      const double t = oracle_eikonal_update(a, b, s[id], dz, dx);
      if (t < T[id]) {
        T[id] = t;
        if (heap_push(&h, t, id)) rc = -1;
      }
    }
  }
  free(h.a);
  free(known);
  return rc;
}
