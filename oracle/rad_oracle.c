/*
 * rad_oracle.c -- plain, slow FP64 CPU oracle for the 3D shape-feature path
 * of PyRadiomics-cuda (arXiv 2510.02894).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's
 * CPU-baseline / reference leg may load this library.  It shares no code,
 * header, table or generator with the CUDA library; neither includes the
 * other.
 *
 * What it computes (paper Sec. 2, "PyRadiomics-cuda design"):
 *   - a marching-cubes triangle mesh of the implicitly zero-padded mask
 *     (Sec. 2, "Marching cubes fused parallel kernels": every cube's eight
 *     corner values are compared against the iso value),
 *   - MeshVolume (signed-tetrahedron sum) and SurfaceArea (triangle-area sum),
 *     both named in Sec. 2 as the features of the first step,
 *   - the maximum 3D diameter and the three planar diameters over the mesh
 *     vertices (Sec. 2, "Parallel diameter calculation": the farthest pair of
 *     vertices, found from all pairs),
 *   - VoxelVolume (count of inside voxels times the voxel volume),
 *   - for a soft probability map: the same mesh with linearly interpolated
 *     iso-0.5 vertices and the analytic FP64 gradient of area, volume and
 *     maximum 3D diameter with respect to every voxel value.
 *
 * The paper prints no lookup table, no triangulation rule and no precision.
 * The readings taken here (face rule, loop orientation, minimum-area
 * triangulation with a lexicographic tie-break, pinned FP64 formulas) are
 * stated beside the code that implements them.  No lookup table is used:
 * every cube's polygons are derived at run time by walking its faces.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction:
 * every formula below is evaluated exactly as written, left to right).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_TOPOLOGY 3

/* ------------------------------------------------------------------ */
/* Voxel grid access (implicit zero padding on every side).            */
/* ------------------------------------------------------------------ */

typedef struct {
  const void* data;
  int kind; /* 0: uint8 mask (inside iff != 0), 1: float32 map, 2: float64 map */
  int64_t nx, ny, nz;
} grid_t;

/* Value of voxel (x,y,z); 0 outside the grid (the implicit padding).
 * A uint8 voxel reads as 1.0 when non-zero so that one iso test (v > 0.5)
 * and one interpolation formula serve both the binary and the soft map:
 * for values 0 and 1 the interpolation parameter is exactly 1/2. */
static double gval(const grid_t* g, int64_t x, int64_t y, int64_t z) {
  if (x < 0 || y < 0 || z < 0 || x >= g->nx || y >= g->ny || z >= g->nz) return 0.0;
  int64_t i = (z * g->ny + y) * g->nx + x;
  if (g->kind == 0) return ((const uint8_t*)g->data)[i] != 0 ? 1.0 : 0.0;
  if (g->kind == 1) return (double)((const float*)g->data)[i];
  return ((const double*)g->data)[i];
}

/* Inside test: value strictly above the iso level 1/2. */
static int is_in(double v) { return v > 0.5; }

/* ------------------------------------------------------------------ */
/* Growable arrays.                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
  void* p;
  int64_t n, cap;
  size_t elem;
} vec_t;

static int vec_push(vec_t* v, const void* item) {
  if (v->n == v->cap) {
    int64_t nc = v->cap ? v->cap * 2 : 1024;
    void* np = realloc(v->p, (size_t)nc * v->elem);
    if (!np) return ORC_ERR_OOM;
    v->p = np;
    v->cap = nc;
  }
  memcpy((char*)v->p + (size_t)v->n * v->elem, item, v->elem);
  v->n++;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Mesh result.                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t nv, nt, nvox;
  int32_t* owner; /* nv x 3: lower grid point of the crossing edge, each in [-1, n-1] */
  int32_t* axis;  /* nv: axis of the crossing edge (0 = x, 1 = y, 2 = z) */
  double* t;      /* nv: iso crossing parameter measured from the owner point */
  double* v0;     /* nv: value at the owner point */
  double* v1;     /* nv: value at the other end of the edge */
  double* u;      /* nv x 3: index-space vertex position (owner + t along axis) */
  int32_t* tri;   /* nt x 3: vertex ids, outward counter-clockwise */
  double volume, area;
  int max_loop;   /* largest polygon met (diagnostic) */
  int64_t n_loops;
  int64_t n_ties; /* loops whose minimum-area choice was decided by the tie-break */
  double spacing[3];
  int64_t dims[3];
} orc_mesh;

/* Canonical vertex key: (z, y, x, axis) of the owner, lexicographic.  Vertex
 * ids are the ranks of these keys, so they follow the canonical order. */
static int64_t vkey(const grid_t* g, int64_t x, int64_t y, int64_t z, int a) {
  return (((z + 1) * (g->ny + 1) + (y + 1)) * (g->nx + 1) + (x + 1)) * 3 + a;
}

static int64_t find_key(const int64_t* keys, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (keys[mid] == key) return mid;
    if (keys[mid] < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

/* ------------------------------------------------------------------ */
/* Cube geometry: corners c = cx + 2 cy + 4 cz; an edge is (corner with  */
/* the axis bit clear, axis).  Local edge ids follow (cz, cy, cx, axis), */
/* which is the global canonical order restricted to one cube.          */
/* ------------------------------------------------------------------ */

static int g_local_edge_id[8][3]; /* -1 where the axis bit of the corner is set */
static int g_local_edge_corner[12], g_local_edge_axis[12];
static int g_tables_ready = 0;

static void init_local_edges(void) {
  if (g_tables_ready) return;
  int n = 0;
  for (int c = 0; c < 8; ++c)
    for (int a = 0; a < 3; ++a) {
      if ((c >> a) & 1) {
        g_local_edge_id[c][a] = -1;
      } else {
        g_local_edge_id[c][a] = n;
        g_local_edge_corner[n] = c;
        g_local_edge_axis[n] = a;
        ++n;
      }
    }
  g_tables_ready = 1;
}

/* Local edge id of the edge joining corners c1 and c2 (adjacent). */
static int edge_between(int c1, int c2) {
  int d = c1 ^ c2;
  int a = d == 1 ? 0 : (d == 2 ? 1 : 2);
  int lo = (c1 >> a) & 1 ? c2 : c1;
  return g_local_edge_id[lo][a];
}

/* Twice the local position of the midpoint of a local edge (integers 0..2). */
static void edge_mid2(int e, int p[3]) {
  int c = g_local_edge_corner[e], a = g_local_edge_axis[e];
  for (int k = 0; k < 3; ++k) p[k] = 2 * ((c >> k) & 1) + (k == a ? 1 : 0);
}

/* ------------------------------------------------------------------ */
/* Triangulations of a k-gon, enumerated once per k (k <= 12).         */
/* Each triangulation is k-2 triples of polygon positions (i < m < j),  */
/* which keeps the polygon's orientation.                               */
/* ------------------------------------------------------------------ */

#define ORC_MAXK 12
typedef struct {
  int count;
  int* tri; /* count x (k-2) x 3 */
} tri_list_t;
static tri_list_t g_tris[ORC_MAXK + 1];

typedef struct {
  int k;
  int pend[ORC_MAXK][2];
  int npend;
  int cur[ORC_MAXK][3];
  int ncur;
  vec_t* out;
} enum_state;

static void enum_rec(enum_state* s) {
  if (s->npend == 0) {
    for (int t = 0; t < s->ncur; ++t)
      for (int q = 0; q < 3; ++q) vec_push(s->out, &s->cur[t][q]);
    return;
  }
  /* take the last pending sub-polygon (i..j); its edge (i,j) lies in exactly
   * one triangle (i,m,j) of any triangulation: enumerate the apex m. */
  int i = s->pend[s->npend - 1][0], j = s->pend[s->npend - 1][1];
  s->npend--;
  for (int m = i + 1; m < j; ++m) {
    int save_np = s->npend, save_nc = s->ncur;
    s->cur[s->ncur][0] = i;
    s->cur[s->ncur][1] = m;
    s->cur[s->ncur][2] = j;
    s->ncur++;
    if (m - i >= 2) { s->pend[s->npend][0] = i; s->pend[s->npend][1] = m; s->npend++; }
    if (j - m >= 2) { s->pend[s->npend][0] = m; s->pend[s->npend][1] = j; s->npend++; }
    enum_rec(s);
    s->npend = save_np;
    s->ncur = save_nc;
  }
  s->pend[s->npend][0] = i;
  s->pend[s->npend][1] = j;
  s->npend++;
}

static int get_triangulations(int k, tri_list_t** out) {
  if (k < 3 || k > ORC_MAXK) return ORC_ERR_TOPOLOGY;
  if (!g_tris[k].tri) {
    vec_t v = {0, 0, 0, sizeof(int)};
    enum_state s;
    memset(&s, 0, sizeof(s));
    s.k = k;
    s.out = &v;
    s.pend[0][0] = 0;
    s.pend[0][1] = k - 1;
    s.npend = 1;
    enum_rec(&s);
    g_tris[k].count = (int)(v.n / (3 * (k - 2)));
    g_tris[k].tri = (int*)v.p;
  }
  *out = &g_tris[k];
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Pinned per-loop triangulation score.                                 */
/*                                                                     */
/* Reading (the paper gives no rule for polygons of 4+ vertices): each  */
/* loop is split into the admissible triangulation (see admissible())   */
/* of minimum total area.  Area is                                      */
/* evaluated in cube-local physical coordinates with this exact FP64    */
/* sequence, so that any other implementation of the same formula makes */
/* the same choice bit for bit:                                         */
/*   local position  w_k = (corner_k + [k == axis] t) * s_k             */
/*   triangle (A,B,C) = canonical rotation (smallest vertex id first)   */
/*   e1 = B - A, e2 = C - A; n = e1 x e2 (each component as a*b - c*d)   */
/*   r = sqrt((n_x^2 + n_y^2) + n_z^2)                                  */
/*   score = sum of r over the triangles in ascending canonical order.  */
/* Area ties go to the larger enclosed volume (tri_vol6), and remaining */
/* ties to the lexicographically smallest sorted list of canonical      */
/* triples (choose_triangulation).                                      */
/* ------------------------------------------------------------------ */

static void canon_triple(int a, int b, int c, int out[3]) {
  /* rotate (keeping orientation) so that the smallest id comes first */
  if (a < b && a < c) { out[0] = a; out[1] = b; out[2] = c; }
  else if (b < a && b < c) { out[0] = b; out[1] = c; out[2] = a; }
  else { out[0] = c; out[1] = a; out[2] = b; }
}

static int cmp_triple(const void* x, const void* y) {
  const int* a = (const int*)x;
  const int* b = (const int*)y;
  for (int q = 0; q < 3; ++q)
    if (a[q] != b[q]) return a[q] < b[q] ? -1 : 1;
  return 0;
}

static double tri_r(const double A[3], const double B[3], const double C[3]) {
  double e1x = B[0] - A[0], e1y = B[1] - A[1], e1z = B[2] - A[2];
  double e2x = C[0] - A[0], e2y = C[1] - A[1], e2z = C[2] - A[2];
  double p, q;
  p = e1y * e2z; q = e1z * e2y; double nx = p - q;
  p = e1z * e2x; q = e1x * e2z; double ny = p - q;
  p = e1x * e2y; q = e1y * e2x; double nz = p - q;
  double sx = nx * nx, sy = ny * ny, sz = nz * nz;
  double s = sx + sy;
  s = s + sz;
  return sqrt(s);
}

/* 1 if local edges e1 and e2 lie on a common face of the cube.  An edge
 * (corner c, axis a) lies on the two faces (b, bit b of c), b != a. */
static int share_face(int e1, int e2) {
  int c1 = g_local_edge_corner[e1], a1 = g_local_edge_axis[e1];
  int c2 = g_local_edge_corner[e2], a2 = g_local_edge_axis[e2];
  for (int b = 0; b < 3; ++b)
    if (b != a1 && b != a2 && ((c1 >> b) & 1) == ((c2 >> b) & 1)) return 1;
  return 0;
}

/* Admissible triangulation: none of its diagonals (triangle sides that are
 * not loop sides) joins two vertices on a common cube face.  Such a diagonal
 * lies in that face; a loop that crosses one face twice could otherwise be
 * closed by triangles lying flat in the face, and the cube on the other side
 * may do the same, so the two would overlap and the mesh would stop being
 * edge-manifold.  Every loop of every case keeps at least one admissible
 * triangulation (checked by the exhaustive 2x2x2 test). */
static int admissible(const int* loop, int k, const int* T, int nt) {
  for (int t = 0; t < nt; ++t) {
    int p[3] = {T[3 * t], T[3 * t + 1], T[3 * t + 2]};
    for (int s = 0; s < 3; ++s) {
      int x = p[s], y = p[(s + 1) % 3];
      int d = (y - x + k) % k;
      if (d == 1 || d == k - 1) continue;
      if (share_face(loop[x], loop[y])) return 0;
    }
  }
  return 1;
}

/* Outward-signed volume of the cone from the cube-local origin over a
 * triangulation (six times the volume), pinned like the score:
 *   sum over ascending canonical triples (A,B,C) of
 *   ((A_x (B_y C_z - B_z C_y) + A_y (B_z C_x - B_x C_z)) + A_z (B_x C_y - B_y C_x)).
 * Two triangulations of one loop differ in it by the volume enclosed between
 * them, which every isometry of the configuration preserves. */
static double tri_vol6(const double A[3], const double B[3], const double C[3]) {
  double p, q;
  p = B[1] * C[2]; q = B[2] * C[1]; double k0 = p - q;
  p = B[2] * C[0]; q = B[0] * C[2]; double k1 = p - q;
  p = B[0] * C[1]; q = B[1] * C[0]; double k2 = p - q;
  double r = A[0] * k0;
  double r1 = A[1] * k1;
  double r2 = A[2] * k2;
  r = r + r1;
  r = r + r2;
  return r;
}

/* Choose the triangulation of one loop.  loop[] holds local edge ids in loop
 * order, wl[e][k] the cube-local positions.  Writes (k-2) canonical triples
 * of local edge ids to out, sorted ascending.
 *
 * Selection among the admissible triangulations:
 *   1. minimum area score S_min;  tied: S <= S_min + S_min * 1e-12;
 *   2. among the tied, maximum volume V6_max;  tied: V6 >= V6_max - 1e-9 s_x s_y s_z;
 *   3. among those, the lexicographically smallest canonical list.
 * Minimum area alone leaves some hexagons with two equal-area choices of
 * different enclosed volume; step 2 makes MeshVolume (and SurfaceArea)
 * invariant under the cube's symmetries. */
static int choose_triangulation(const int* loop, int k, double wl[12][3], const double sp[3], int* out,
                                int* tie) {
  tri_list_t* tl;
  int st = get_triangulations(k, &tl);
  if (st) return st;
  int nt = k - 2;
  int nc = 0;
  int (*lists)[ORC_MAXK][3] = (int (*)[ORC_MAXK][3])malloc(sizeof(int) * ORC_MAXK * 3 * (size_t)tl->count);
  double* sc = (double*)malloc(sizeof(double) * (size_t)tl->count);
  double* vv = (double*)malloc(sizeof(double) * (size_t)tl->count);
  if (!lists || !sc || !vv) { free(lists); free(sc); free(vv); return ORC_ERR_OOM; }
  for (int c = 0; c < tl->count; ++c) {
    const int* T = tl->tri + (size_t)c * nt * 3;
    if (!admissible(loop, k, T, nt)) continue;
    for (int t = 0; t < nt; ++t)
      canon_triple(loop[T[3 * t]], loop[T[3 * t + 1]], loop[T[3 * t + 2]], lists[nc][t]);
    qsort(lists[nc], (size_t)nt, sizeof(lists[nc][0]), cmp_triple);
    double s = 0.0, v = 0.0;
    for (int t = 0; t < nt; ++t) {
      const int* tr = lists[nc][t];
      s = s + tri_r(wl[tr[0]], wl[tr[1]], wl[tr[2]]);
      v = v + tri_vol6(wl[tr[0]], wl[tr[1]], wl[tr[2]]);
    }
    sc[nc] = s;
    vv[nc] = v;
    ++nc;
  }
  if (nc == 0) { free(lists); free(sc); free(vv); return ORC_ERR_TOPOLOGY; }
  double smin = sc[0];
  for (int c = 1; c < nc; ++c)
    if (sc[c] < smin) smin = sc[c];
  double slim = smin + smin * 1e-12;
  double vmax = 0.0;
  int have = 0, ntied = 0;
  for (int c = 0; c < nc; ++c)
    if (sc[c] <= slim) {
      ++ntied;
      if (!have || vv[c] > vmax) { vmax = vv[c]; have = 1; }
    }
  double vlim = vmax - ((sp[0] * sp[1]) * sp[2]) * 1e-9;
  int best = -1;
  for (int c = 0; c < nc; ++c) {
    if (sc[c] > slim || vv[c] < vlim) continue;
    if (best < 0) { best = c; continue; }
    int lex = 0;
    for (int t = 0; t < nt && lex == 0; ++t) lex = cmp_triple(lists[c][t], lists[best][t]);
    if (lex < 0) best = c;
  }
  *tie = ntied > 1;
  memcpy(out, lists[best], sizeof(int) * 3 * (size_t)nt);
  free(lists); free(sc); free(vv);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Polygons of one cube by walking its faces.                           */
/*                                                                     */
/* Reading of the ambiguous faces (the paper names brute-force marching */
/* cubes, Sec. 2, but no table): on a face whose two inside corners are */
/* diagonal, the inside corners are separated (each is cut off by its   */
/* own segment).  The rule uses only the four face corners, so the two  */
/* cubes sharing a face make the same cut and the mesh is closed.       */
/*                                                                     */
/* Orientation: seen from outside the cube, every segment runs with the */
/* inside corner(s) of its face on its right.  Chained, the loops turn  */
/* counter-clockwise around the normal that points from inside to       */
/* outside, so (b-a) x (c-a) of every triangle points outwards.         */
/* Each loop is closed by its own disk (the cube interior adds no        */
/* tunnels).                                                            */
/* ------------------------------------------------------------------ */

static int cube_loops(const int in[8], int next[12], int loops[12][ORC_MAXK], int loopk[12], int* nloops) {
  for (int e = 0; e < 12; ++e) next[e] = -1;
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    for (int s = 0; s < 2; ++s) {
      int q[4];
      q[0] = (s << a);
      q[1] = (s << a) | (1 << b);
      q[2] = (s << a) | (1 << b) | (1 << c);
      q[3] = (s << a) | (1 << c);
      int nrm[3] = {0, 0, 0};
      nrm[a] = s ? 1 : -1;
      int cross_idx[4], nc = 0;
      for (int i = 0; i < 4; ++i)
        if (in[q[i]] != in[q[(i + 1) % 4]]) cross_idx[nc++] = i;
      int segs[2][3]; /* (face edge i1, face edge i2, reference inside corner) */
      int nseg = 0;
      if (nc == 2) {
        int cin = -1;
        for (int i = 0; i < 4; ++i)
          if (in[q[i]]) { cin = q[i]; break; }
        segs[0][0] = cross_idx[0];
        segs[0][1] = cross_idx[1];
        segs[0][2] = cin;
        nseg = 1;
      } else if (nc == 4) {
        for (int j = 0; j < 4; ++j)
          if (in[q[j]]) {
            segs[nseg][0] = (j + 3) % 4; /* face edge q[j-1] -- q[j] */
            segs[nseg][1] = j;           /* face edge q[j] -- q[j+1] */
            segs[nseg][2] = q[j];
            ++nseg;
          }
      } else if (nc != 0) {
        return ORC_ERR_TOPOLOGY;
      }
      for (int sg = 0; sg < nseg; ++sg) {
        int fe1 = segs[sg][0], fe2 = segs[sg][1], cin = segs[sg][2];
        int e1 = edge_between(q[fe1], q[(fe1 + 1) % 4]);
        int e2 = edge_between(q[fe2], q[(fe2 + 1) % 4]);
        int p1[3], p2[3], w[3], d[3];
        edge_mid2(e1, p1);
        edge_mid2(e2, p2);
        for (int k = 0; k < 3; ++k) {
          d[k] = p2[k] - p1[k];
          w[k] = 2 * ((cin >> k) & 1) - p1[k];
        }
        int cr[3] = {d[1] * w[2] - d[2] * w[1], d[2] * w[0] - d[0] * w[2], d[0] * w[1] - d[1] * w[0]};
        int dot = cr[0] * nrm[0] + cr[1] * nrm[1] + cr[2] * nrm[2];
        if (dot == 0) return ORC_ERR_TOPOLOGY;
        int from = dot < 0 ? e1 : e2, to = dot < 0 ? e2 : e1;
        if (next[from] != -1) return ORC_ERR_TOPOLOGY;
        next[from] = to;
      }
    }
  }
  /* chain the segments into loops, starting each at its smallest local edge */
  int visited[12] = {0};
  *nloops = 0;
  for (int e = 0; e < 12; ++e) {
    if (next[e] < 0 || visited[e]) continue;
    int k = 0, cur = e;
    while (!visited[cur]) {
      if (k >= ORC_MAXK || next[cur] < 0) return ORC_ERR_TOPOLOGY;
      visited[cur] = 1;
      loops[*nloops][k++] = cur;
      cur = next[cur];
    }
    if (cur != e || k < 3) return ORC_ERR_TOPOLOGY;
    loopk[*nloops] = k;
    (*nloops)++;
  }
  return ORC_OK;
}

/* O-relative physical position of a vertex (O = centre of the padded box):
 *   p_k = ((g_k - (n_k - 1)/2) + [k == axis] t) * s_k. */
static void vpos_rel(const orc_mesh* m, int64_t v, double p[3]) {
  for (int k = 0; k < 3; ++k) {
    double base = (double)m->owner[3 * v + k] - (double)(m->dims[k] - 1) * 0.5;
    double tt = (m->axis[v] == k) ? m->t[v] : 0.0;
    p[k] = (base + tt) * m->spacing[k];
  }
}

/* ------------------------------------------------------------------ */
/* Mesh construction.                                                   */
/* ------------------------------------------------------------------ */

void orc_mesh_free(orc_mesh* m) {
  if (!m) return;
  free(m->owner); free(m->axis); free(m->t); free(m->v0); free(m->v1); free(m->u); free(m->tri);
  free(m);
}

/* Build the mesh of a uint8 mask (kind 0) or a float32 / float64 map
 * (kinds 1, 2).  data is C-order [nz][ny][nx], x fastest. */
orc_mesh* orc_mesh_build(const void* data, int kind, int64_t nx, int64_t ny, int64_t nz,
                         const double spacing[3], int* status) {
  *status = ORC_OK;
  init_local_edges();
  if (!data || nx <= 0 || ny <= 0 || nz <= 0 || kind < 0 || kind > 2) { *status = ORC_ERR_ARG; return NULL; }
  grid_t g = {data, kind, nx, ny, nz};
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  if (!m) { *status = ORC_ERR_OOM; return NULL; }
  m->dims[0] = nx; m->dims[1] = ny; m->dims[2] = nz;
  for (int k = 0; k < 3; ++k) m->spacing[k] = spacing[k];

  /* 1. vertices: one per grid edge whose endpoints differ in inside-ness,
   *    in canonical (z, y, x, axis) order of the lower endpoint. */
  vec_t keys = {0, 0, 0, sizeof(int64_t)};
  vec_t own = {0, 0, 0, sizeof(int32_t) * 3};
  vec_t ax = {0, 0, 0, sizeof(int32_t)};
  vec_t tv = {0, 0, 0, sizeof(double)};
  vec_t v0v = {0, 0, 0, sizeof(double)};
  vec_t v1v = {0, 0, 0, sizeof(double)};
  int64_t nvox = 0;
  for (int64_t z = -1; z < nz; ++z)
    for (int64_t y = -1; y < ny; ++y)
      for (int64_t x = -1; x < nx; ++x) {
        double a0 = gval(&g, x, y, z);
        if (x >= 0 && y >= 0 && z >= 0 && is_in(a0)) ++nvox;
        for (int a = 0; a < 3; ++a) {
          double a1 = gval(&g, x + (a == 0), y + (a == 1), z + (a == 2));
          if (is_in(a0) == is_in(a1)) continue;
          int64_t key = vkey(&g, x, y, z, a);
          int32_t o[3] = {(int32_t)x, (int32_t)y, (int32_t)z};
          int32_t aa = a;
          /* linear interpolation at the iso level 1/2 (exactly 1/2 for 0/1 values) */
          double tt = (0.5 - a0) / (a1 - a0);
          if (vec_push(&keys, &key) || vec_push(&own, o) || vec_push(&ax, &aa) ||
              vec_push(&tv, &tt) || vec_push(&v0v, &a0) || vec_push(&v1v, &a1)) {
            *status = ORC_ERR_OOM;
            goto fail;
          }
        }
      }
  m->nv = keys.n;
  m->nvox = nvox;
  m->owner = (int32_t*)own.p; own.p = NULL;
  m->axis = (int32_t*)ax.p; ax.p = NULL;
  m->t = (double*)tv.p; tv.p = NULL;
  m->v0 = (double*)v0v.p; v0v.p = NULL;
  m->v1 = (double*)v1v.p; v1v.p = NULL;
  m->u = (double*)malloc(sizeof(double) * 3 * (size_t)(m->nv ? m->nv : 1));
  if (!m->u) { *status = ORC_ERR_OOM; goto fail; }
  for (int64_t v = 0; v < m->nv; ++v)
    for (int k = 0; k < 3; ++k)
      m->u[3 * v + k] = (double)m->owner[3 * v + k] + (m->axis[v] == k ? m->t[v] : 0.0);

  /* 2. triangles: every cube of the padded grid (lower corner in [-1, n-1]^3),
   *    in (z, y, x) order; within a cube, the triangles sorted by canonical
   *    triple. */
  vec_t tris = {0, 0, 0, sizeof(int32_t) * 3};
  double vol = 0.0, area = 0.0;
  for (int64_t z = -1; z < nz; ++z)
    for (int64_t y = -1; y < ny; ++y)
      for (int64_t x = -1; x < nx; ++x) {
        int in[8], nin = 0;
        double cv[8];
        for (int c = 0; c < 8; ++c) {
          cv[c] = gval(&g, x + (c & 1), y + ((c >> 1) & 1), z + ((c >> 2) & 1));
          in[c] = is_in(cv[c]);
          nin += in[c];
        }
        if (nin == 0 || nin == 8) continue;
        int next[12], loops[12][ORC_MAXK], loopk[12], nl;
        int st = cube_loops(in, next, loops, loopk, &nl);
        if (st) { *status = st; free(tris.p); goto fail; }
        /* global ids and cube-local positions of the crossing edges */
        int64_t gid[12];
        double wl[12][3];
        for (int e = 0; e < 12; ++e) {
          if (next[e] < 0) continue;
          int c = g_local_edge_corner[e], a = g_local_edge_axis[e];
          int64_t ox = x + (c & 1), oy = y + ((c >> 1) & 1), oz = z + ((c >> 2) & 1);
          gid[e] = find_key((const int64_t*)keys.p, keys.n, vkey(&g, ox, oy, oz, a));
          if (gid[e] < 0) { *status = ORC_ERR_TOPOLOGY; free(tris.p); goto fail; }
          double tt = m->t[gid[e]];
          for (int k = 0; k < 3; ++k) {
            double corner = (double)((c >> k) & 1);
            double add = (k == a) ? tt : 0.0;
            wl[e][k] = (corner + add) * spacing[k];
          }
        }
        int ctri[ORC_MAXK * 12][3], nct = 0;
        for (int l = 0; l < nl; ++l) {
          int k = loopk[l], tie = 0;
          if (k > m->max_loop) m->max_loop = k;
          m->n_loops++;
          int chosen[ORC_MAXK][3];
          st = choose_triangulation(loops[l], k, wl, spacing, &chosen[0][0], &tie);
          if (st) { *status = st; free(tris.p); goto fail; }
          m->n_ties += tie;
          for (int t = 0; t < k - 2; ++t) {
            ctri[nct][0] = chosen[t][0];
            ctri[nct][1] = chosen[t][1];
            ctri[nct][2] = chosen[t][2];
            ++nct;
          }
        }
        qsort(ctri, (size_t)nct, sizeof(ctri[0]), cmp_triple);
        for (int t = 0; t < nct; ++t) {
          int32_t tr[3] = {(int32_t)gid[ctri[t][0]], (int32_t)gid[ctri[t][1]], (int32_t)gid[ctri[t][2]]};
          if (vec_push(&tris, tr)) { *status = ORC_ERR_OOM; free(tris.p); goto fail; }
          /* MeshVolume: signed tetrahedron (O, a, b, c) = a . (b x c) / 6;
           * SurfaceArea: |(b - a) x (c - a)| / 2 (Sec. 2, computed on the fly). */
          double pa[3], pb[3], pc[3];
          vpos_rel(m, tr[0], pa);
          vpos_rel(m, tr[1], pb);
          vpos_rel(m, tr[2], pc);
          double bxc0 = pb[1] * pc[2] - pb[2] * pc[1];
          double bxc1 = pb[2] * pc[0] - pb[0] * pc[2];
          double bxc2 = pb[0] * pc[1] - pb[1] * pc[0];
          double tv6 = (pa[0] * bxc0 + pa[1] * bxc1 + pa[2] * bxc2) / 6.0;
          vol = vol + tv6;
          area = area + 0.5 * tri_r(pa, pb, pc);
        }
      }
  m->nt = tris.n;
  m->tri = (int32_t*)tris.p;
  m->volume = vol;
  m->area = area;
  free(keys.p);
  return m;
fail:
  free(keys.p); free(own.p); free(ax.p); free(tv.p); free(v0v.p); free(v1v.p);
  orc_mesh_free(m);
  return NULL;
}

/* Accessors for the ctypes wrapper. */
int64_t orc_mesh_nv(const orc_mesh* m) { return m->nv; }
int64_t orc_mesh_nt(const orc_mesh* m) { return m->nt; }
int64_t orc_mesh_nvox(const orc_mesh* m) { return m->nvox; }
double orc_mesh_volume(const orc_mesh* m) { return m->volume; }
double orc_mesh_area(const orc_mesh* m) { return m->area; }
int orc_mesh_max_loop(const orc_mesh* m) { return m->max_loop; }
int64_t orc_mesh_n_ties(const orc_mesh* m) { return m->n_ties; }
void orc_mesh_copy(const orc_mesh* m, int32_t* owner, int32_t* axis, double* t, double* u, int32_t* tri) {
  if (owner) memcpy(owner, m->owner, sizeof(int32_t) * 3 * (size_t)m->nv);
  if (axis) memcpy(axis, m->axis, sizeof(int32_t) * (size_t)m->nv);
  if (t) memcpy(t, m->t, sizeof(double) * (size_t)m->nv);
  if (u) memcpy(u, m->u, sizeof(double) * 3 * (size_t)m->nv);
  if (tri) memcpy(tri, m->tri, sizeof(int32_t) * 3 * (size_t)m->nt);
}

/* ------------------------------------------------------------------ */
/* Diameters (Sec. 2, "Parallel diameter calculation").                */
/*                                                                     */
/* Pinned squared distance of vertices i and j (index positions u,     */
/* spacing s), evaluated left to right in FP64 with no contraction:     */
/*   D_k = (u_ik - u_jk) * s_k                                          */
/*   d2  = ((D_x * D_x + D_y * D_y) + D_z * D_z)                        */
/* Diameter = sqrt(max d2) (correctly rounded).  Argmax = smallest      */
/* (i, j), i < j, among the pairs attaining the maximum.  The planar    */
/* diameters restrict to pairs with exactly equal z (Slice, the XY      */
/* plane), y (Column, XZ) or x (Row, YZ) coordinate.                     */
/* ------------------------------------------------------------------ */

static double pin_d2(const double* u, int64_t i, int64_t j, const double s[3]) {
  double dx = u[3 * i] - u[3 * j];
  double dy = u[3 * i + 1] - u[3 * j + 1];
  double dz = u[3 * i + 2] - u[3 * j + 2];
  dx = dx * s[0];
  dy = dy * s[1];
  dz = dz * s[2];
  double xx = dx * dx, yy = dy * dy, zz = dz * dz;
  double r = xx + yy;
  r = r + zz;
  return r;
}

double orc_pair_d2(const double* u, int64_t i, int64_t j, const double s[3]) { return pin_d2(u, i, j, s); }

typedef struct {
  double d2;
  int64_t i, j;
} best_t;

static int better(double d2, int64_t i, int64_t j, const best_t* b) {
  if (b->i < 0) return 1;
  if (d2 != b->d2) return d2 > b->d2;
  if (i != b->i) return i < b->i;
  return j < b->j;
}

static void take(best_t* b, double d2, int64_t i, int64_t j) {
  if (better(d2, i, j, b)) { b->d2 = d2; b->i = i; b->j = j; }
}

/* Brute force over all pairs i < j: out[0] 3D, out[1] Slice (equal z),
 * out[2] Column (equal y), out[3] Row (equal x).  d2 = 0 and (-1, -1) where
 * no pair exists.  Threads split the outer loop; the per-thread results are
 * merged under the same total order, so the result does not depend on the
 * thread count. */
int orc_diameters_bruteforce(const double* u, int64_t n, const double s[3], double d2_out[4],
                             int64_t i_out[4], int64_t j_out[4]) {
  best_t gb[4];
  for (int q = 0; q < 4; ++q) { gb[q].d2 = 0.0; gb[q].i = -1; gb[q].j = -1; }
#pragma omp parallel
  {
    best_t lb[4];
    for (int q = 0; q < 4; ++q) { lb[q].d2 = 0.0; lb[q].i = -1; lb[q].j = -1; }
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = i + 1; j < n; ++j) {
        double d2 = pin_d2(u, i, j, s);
        take(&lb[0], d2, i, j);
        if (u[3 * i + 2] == u[3 * j + 2]) take(&lb[1], d2, i, j);
        if (u[3 * i + 1] == u[3 * j + 1]) take(&lb[2], d2, i, j);
        if (u[3 * i + 0] == u[3 * j + 0]) take(&lb[3], d2, i, j);
      }
    }
#pragma omp critical
    {
      for (int q = 0; q < 4; ++q)
        if (lb[q].i >= 0) take(&gb[q], lb[q].d2, lb[q].i, lb[q].j);
    }
  }
  for (int q = 0; q < 4; ++q) { d2_out[q] = gb[q].d2; i_out[q] = gb[q].i; j_out[q] = gb[q].j; }
  return ORC_OK;
}

/* Brute force over the pairs of an explicit subset (ids ascending). */
static void subset_max(const double* u, const int64_t* ids, int64_t m, const double s[3], best_t* out) {
  best_t gb = {0.0, -1, -1};
#pragma omp parallel
  {
    best_t lb = {0.0, -1, -1};
#pragma omp for schedule(dynamic, 16)
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = a + 1; b < m; ++b) take(&lb, pin_d2(u, ids[a], ids[b], s), ids[a], ids[b]);
#pragma omp critical
    {
      if (lb.i >= 0) take(&gb, lb.d2, lb.i, lb.j);
    }
  }
  *out = gb;
}

/* Brute force over the pairs of a caller-given vertex subset (ids
 * ascending); used with a candidate set that provably holds every vertex of
 * every maximal pair (see oracle/__init__.py). */
int orc_subset_max(const double* u, const int64_t* ids, int64_t m, const double s[3], double* d2_out,
                   int64_t* i_out, int64_t* j_out) {
  best_t bb;
  subset_max(u, ids, m, s, &bb);
  *d2_out = bb.i >= 0 ? bb.d2 : 0.0;
  *i_out = bb.i;
  *j_out = bb.j;
  return ORC_OK;
}

/* Maximum 3D diameter with an exact pruning step (same result as the brute
 * force, for large meshes):
 *   1. L = d2 of an actual pair (two farthest-point sweeps from vertex 0):
 *      a lower bound of the maximum.
 *   2. Every pair (i, j) satisfies d2(i, j) <= U_i, the squared distance from
 *      i to the farthest corner of the vertices' bounding box.  A vertex with
 *      U_i (1 + 1e-9) < L can belong to no pair reaching L (the factor covers
 *      the rounding of both formulas), so it is dropped.
 *   3. Brute force over the pairs of the remaining vertices. */
int orc_diameter3d_pruned(const double* u, int64_t n, const double s[3], double* d2_out, int64_t* i_out,
                          int64_t* j_out, int64_t* n_kept) {
  *d2_out = 0.0; *i_out = -1; *j_out = -1; *n_kept = 0;
  if (n < 2) return ORC_OK;
  int64_t a = 0, b = 0;
  for (int sweep = 0; sweep < 2; ++sweep) {
    int64_t far = a;
    double fd = -1.0;
    for (int64_t j = 0; j < n; ++j) {
      double d2 = pin_d2(u, a, j, s);
      if (d2 > fd) { fd = d2; far = j; }
    }
    b = a;
    a = far;
  }
  double L = pin_d2(u, a, b, s);
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) { lo[k] = u[k]; hi[k] = u[k]; }
  for (int64_t v = 1; v < n; ++v)
    for (int k = 0; k < 3; ++k) {
      if (u[3 * v + k] < lo[k]) lo[k] = u[3 * v + k];
      if (u[3 * v + k] > hi[k]) hi[k] = u[3 * v + k];
    }
  int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!ids) return ORC_ERR_OOM;
  int64_t m = 0;
  for (int64_t v = 0; v < n; ++v) {
    double U = 0.0;
    for (int k = 0; k < 3; ++k) {
      double d1 = (u[3 * v + k] - lo[k]) * s[k], d2 = (hi[k] - u[3 * v + k]) * s[k];
      double dd = d1 > d2 ? d1 : d2;
      U = U + dd * dd;
    }
    if (U * (1.0 + 1e-9) >= L) ids[m++] = v;
  }
  best_t bb;
  subset_max(u, ids, m, s, &bb);
  free(ids);
  *d2_out = bb.i >= 0 ? bb.d2 : 0.0;
  *i_out = bb.i;
  *j_out = bb.j;
  *n_kept = m;
  return ORC_OK;
}

/* Planar diameter: group the vertices by their exact coordinate on `axis`
 * (2: Slice, 1: Column, 0: Row) and brute-force every group.  Same result as
 * the filtered brute force above. */
typedef struct {
  double key;
  int64_t id;
} keyid_t;

static int cmp_keyid(const void* x, const void* y) {
  const keyid_t* a = (const keyid_t*)x;
  const keyid_t* b = (const keyid_t*)y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

int orc_diameter2d_grouped(const double* u, int64_t n, const double s[3], int axis, double* d2_out,
                           int64_t* i_out, int64_t* j_out) {
  *d2_out = 0.0; *i_out = -1; *j_out = -1;
  if (axis < 0 || axis > 2) return ORC_ERR_ARG;
  if (n < 2) return ORC_OK;
  keyid_t* kv = (keyid_t*)malloc(sizeof(keyid_t) * (size_t)n);
  int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!kv || !ids) { free(kv); free(ids); return ORC_ERR_OOM; }
  for (int64_t v = 0; v < n; ++v) { kv[v].key = u[3 * v + axis]; kv[v].id = v; }
  qsort(kv, (size_t)n, sizeof(keyid_t), cmp_keyid);
  best_t gb = {0.0, -1, -1};
  int64_t beg = 0;
  while (beg < n) {
    int64_t end = beg + 1;
    while (end < n && kv[end].key == kv[beg].key) ++end;
    if (end - beg >= 2) {
      for (int64_t q = beg; q < end; ++q) ids[q - beg] = kv[q].id;
      best_t bb;
      subset_max(u, ids, end - beg, s, &bb);
      if (bb.i >= 0) take(&gb, bb.d2, bb.i, bb.j);
    }
    beg = end;
  }
  free(kv);
  free(ids);
  *d2_out = gb.i >= 0 ? gb.d2 : 0.0;
  *i_out = gb.i;
  *j_out = gb.j;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Soft map: analytic FP64 gradient of L = gA * A + gV * V + gD * D3    */
/* with respect to every voxel value (chain rule through the vertex     */
/* interpolation t = (1/2 - v0) / (v1 - v0); the mesh topology and the   */
/* triangulation choice are held fixed, the diameter uses the           */
/* tie-broken argmax pair).                                             */
/*   dA/da = (b - c) x n^ / 2, dA/db = (c - a) x n^ / 2,                */
/*   dA/dc = (a - b) x n^ / 2              (n^ = unit triangle normal)  */
/*   dV/da = (b x c) / 6, dV/db = (c x a) / 6, dV/dc = (a x b) / 6     */
/*   dD/dp_i = (p_i - p_j) / D, dD/dp_j = -(p_i - p_j) / D             */
/*   dp_axis/dt = s_axis                                                */
/*   dt/dv0 = (1/2 - v1) / (v1 - v0)^2, dt/dv1 = -(1/2 - v0) / (v1 - v0)^2 */
/* grad is dense [nz][ny][nx] float64; argmax pair (i3, j3) from the     */
/* diameter routines (pass -1 to leave the diameter term out).          */
/* ------------------------------------------------------------------ */

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* The same with the planar diameters too: gD[q] and the argmax pair
 * (pairs[2q], pairs[2q + 1]) for q = 0 (3D), 1 (Slice), 2 (Column), 3 (Row).
 * Each diameter term is the 3D term's formula on its own pair (the pair, and
 * so the plane, held fixed). */
int orc_soft_grad4(const orc_mesh* m, double gA, double gV, const double gD[4], const int64_t pairs[8], double* grad);

int orc_soft_grad(const orc_mesh* m, double gA, double gV, double gD, int64_t i3, int64_t j3, double* grad) {
  const double g4[4] = {gD, 0.0, 0.0, 0.0};
  const int64_t p4[8] = {i3, j3, -1, -1, -1, -1, -1, -1};
  return orc_soft_grad4(m, gA, gV, g4, p4, grad);
}

int orc_soft_grad4(const orc_mesh* m, double gA, double gV, const double gD[4], const int64_t pairs[8], double* grad) {
  int64_t nvox = m->dims[0] * m->dims[1] * m->dims[2];
  memset(grad, 0, sizeof(double) * (size_t)nvox);
  double* gp = (double*)calloc((size_t)(m->nv ? m->nv : 1) * 3, sizeof(double));
  if (!gp) return ORC_ERR_OOM;
  for (int64_t t = 0; t < m->nt; ++t) {
    int32_t ia = m->tri[3 * t], ib = m->tri[3 * t + 1], ic = m->tri[3 * t + 2];
    double a[3], b[3], c[3];
    vpos_rel(m, ia, a);
    vpos_rel(m, ib, b);
    vpos_rel(m, ic, c);
    double e1[3], e2[3], n[3];
    for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; }
    cross3(e1, e2, n);
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (nn > 0.0) {
      double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
      double bc[3], ca[3], ab[3], ga[3], gb[3], gc[3];
      for (int k = 0; k < 3; ++k) { bc[k] = b[k] - c[k]; ca[k] = c[k] - a[k]; ab[k] = a[k] - b[k]; }
      cross3(bc, nh, ga);
      cross3(ca, nh, gb);
      cross3(ab, nh, gc);
      for (int k = 0; k < 3; ++k) {
        gp[3 * ia + k] += gA * 0.5 * ga[k];
        gp[3 * ib + k] += gA * 0.5 * gb[k];
        gp[3 * ic + k] += gA * 0.5 * gc[k];
      }
    }
    double vbc[3], vca[3], vab[3];
    cross3(b, c, vbc);
    cross3(c, a, vca);
    cross3(a, b, vab);
    for (int k = 0; k < 3; ++k) {
      gp[3 * ia + k] += gV * vbc[k] / 6.0;
      gp[3 * ib + k] += gV * vca[k] / 6.0;
      gp[3 * ic + k] += gV * vab[k] / 6.0;
    }
  }
  for (int q = 0; q < 4; ++q) {
    const int64_t i3 = pairs[2 * q], j3 = pairs[2 * q + 1];
    if (i3 < 0 || j3 < 0 || gD[q] == 0.0) continue;
    double pi[3], pj[3], d[3];
    vpos_rel(m, i3, pi);
    vpos_rel(m, j3, pj);
    for (int k = 0; k < 3; ++k) d[k] = pi[k] - pj[k];
    double D = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (D > 0.0)
      for (int k = 0; k < 3; ++k) {
        gp[3 * i3 + k] += gD[q] * d[k] / D;
        gp[3 * j3 + k] -= gD[q] * d[k] / D;
      }
  }
  for (int64_t v = 0; v < m->nv; ++v) {
    int a = m->axis[v];
    double dLdt = gp[3 * v + a] * m->spacing[a];
    double v0 = m->v0[v], v1 = m->v1[v];
    double den = (v1 - v0) * (v1 - v0);
    double d0 = (0.5 - v1) / den, d1 = -(0.5 - v0) / den;
    int64_t x = m->owner[3 * v], y = m->owner[3 * v + 1], z = m->owner[3 * v + 2];
    if (x >= 0 && y >= 0 && z >= 0 && x < m->dims[0] && y < m->dims[1] && z < m->dims[2])
      grad[(z * m->dims[1] + y) * m->dims[0] + x] += dLdt * d0;
    int64_t x1 = x + (a == 0), y1 = y + (a == 1), z1 = z + (a == 2);
    if (x1 >= 0 && y1 >= 0 && z1 >= 0 && x1 < m->dims[0] && y1 < m->dims[1] && z1 < m->dims[2])
      grad[(z1 * m->dims[1] + y1) * m->dims[0] + x1] += dLdt * d1;
  }
  free(gp);
  return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
