// C ABI of the compressed-vector library: argument checks, format set-up,
// per-format trigonometric tables, launch shapes, batched plans and the
// launch-shape tuner.  Kernels live in ivc_ops.cu and ivc_baseline.cu.
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ivc_internal.h"

using namespace ivc;

namespace {

const long double kPiL = 3.14159265358979323846264338327950288419716939937510L;
// node counts of the tanh map's encoder tables: |theta| in [0, pi], phi in
// [0, pi/2] at spacing pi / 1024
constexpr int kTanhEstT = 1025, kTanhEstP = 513;

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ------------------------------------------------------------ format set-up

struct Geometry {
  int N, M;
};

ivc_status geometry(const ivc_format *f, Geometry *g) {
  if (!f) return IVC_ERR_ARG;
  const int total = f->sign_bits + f->exp_bits + f->man_bits + f->phi_bits + f->theta_bits;
  if (f->sign_bits < 0 || f->sign_bits > 1 || f->exp_bits < 2 || f->exp_bits > 8 ||
      f->man_bits < 1 || f->man_bits > 23 || f->phi_bits < 1 || f->theta_bits < 1 ||
      total > 64 || f->reserved != 0 || f->underflow_mode < 0 || f->underflow_mode > 1 ||
      f->overflow_mode < 0 || f->overflow_mode > 1)
    return IVC_ERR_FORMAT;
  // every normal exponent field must map to a normal FP32 exponent
  const int emaxn = (1 << f->exp_bits) - 2;
  const int e_off = f->exp_bias - 127;
  if (1 - e_off < 1 || emaxn - e_off > 254) return IVC_ERR_FORMAT;
  long long N, M;
  if (f->map == IVC_MAP_FRACSPLIT) {
    const int P = f->phi_bits + f->theta_bits;
    if (P > 40 || f->nphi_max_p1 < 2) return IVC_ERR_FORMAT;
    M = f->nphi_max_p1 - 1;
    N = ((long long)1 << P) / f->nphi_max_p1 - 1;
  } else if (f->map == IVC_MAP_UNIFORM || f->map == IVC_MAP_TANH) {
    if (f->theta_bits > 19 || f->phi_bits > 18) return IVC_ERR_FORMAT;
    N = (1LL << f->theta_bits) - 1;
    M = (1LL << f->phi_bits) - 1;
    if (f->map == IVC_MAP_TANH && !(f->gamma > 0.0 && f->gamma < 20.0)) return IVC_ERR_FORMAT;
  } else {
    return IVC_ERR_FORMAT;
  }
  if (N < 1 || M < 1 || N >= (1LL << 19) || M >= (1LL << 18)) return IVC_ERR_FORMAT;
  g->N = (int)N;
  g->M = (int)M;
  return IVC_OK;
}

void ff_split(long double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (long double)h);
}

TabEntry entry_of(long double c, long double s) {
  TabEntry e;
  ff_split(c, e.ch, e.cl);
  ff_split(s, e.sh, e.sl);
  return e;
}

// Head-table geometry of the folded grid pi b / (2D), b in [0, D/2]: entries at
// b = i 2^s, the remainder rounded to the nearest entry; s is the smallest step
// with at most 1024 entries.
int table_entries(int D, int s) {
  return s == 0 ? D / 2 + 1 : ((D / 2 + (1 << (s - 1))) >> s) + 1;
}

int table_shift(int D) {
  int s = 0;
  while (table_entries(D, s) > 1024) ++s;
  return s;
}

void uniform_table(int D, std::vector<TabEntry> &out) {
  const int s = table_shift(D);
  const int nent = table_entries(D, s);
  for (int i = 0; i < nent; ++i) {
    if (i == 0) {
      out.push_back(TabEntry{1.0f, 0.0f, 0.0f, 0.0f});
      continue;
    }
    const long double a = kPiL * (long double)((long long)i << s) / (2.0L * D);
    out.push_back(entry_of(cosl(a), sinl(a)));
  }
}

// tanh companding (Sec. 2.5): psi^ of code n and psi at boundary t.
long double psi_of_t(long double t, long double nmax, long double g) {
  const long double c = tanhl(g);
  return 0.5L * (1.0L + atanhl(c * (2.0L * t / nmax - 1.0L)) / g);
}

TabEntry theta_entry_psi(long double psi) {  // theta = pi (2 psi - 1)
  if (psi == 0.5L) return TabEntry{1.0f, 0.0f, 0.0f, 0.0f};
  if (psi == 0.0L || psi == 1.0L) return TabEntry{-1.0f, 0.0f, 0.0f, 0.0f};
  const long double th = kPiL * (2.0L * psi - 1.0L);
  return entry_of(cosl(th), sinl(th));
}

TabEntry phi_entry_psi(long double psi) {  // phi = pi psi
  if (psi == 0.0L) return TabEntry{1.0f, 0.0f, 0.0f, 0.0f};
  if (psi == 1.0L) return TabEntry{-1.0f, 0.0f, 0.0f, 0.0f};
  if (psi == 0.5L) return TabEntry{0.0f, 0.0f, 1.0f, 0.0f};
  const long double ph = kPiL * psi;
  return entry_of(cosl(ph), sinl(ph));
}

struct TableKey {
  int device, map, N, M;
  double gamma;
  bool operator<(const TableKey &o) const {
    return std::tie(device, map, N, M, gamma) < std::tie(o.device, o.map, o.N, o.M, o.gamma);
  }
};

struct TableSet {
  TabEntry *dev = nullptr;
  size_t n_uniform_t = 0, n_uniform_p = 0, off_phi = 0;
  size_t off_dec_t = 0, off_dec_p = 0, off_bnd_t = 0, off_bnd_p = 0, off_est = 0;
};

// Node tables of the tanh map's fast encoder (Sec. 2.5, reading R11): the bin
// coordinate t(a) = n_max (tanh(g w(a)) + c) / (2c), c = tanh g, with
// w = a / pi for |theta| = a in [0, pi] (t from n_max / 2 to n_max) and
// w = 2 a / pi - 1 for phi = a in [0, pi/2] (t from 0 to n_max / 2), at the
// nodes a = j pi / 1024: floor t, the fraction, t' and t'' / 2 (derivatives
// in the angle), for a quadratic step to the input angle.
void tanh_est_table(long double nmax, long double g, bool theta, int nodes,
                    std::vector<TabEntry> &out) {
  const long double c = tanhl(g);
  const long double s = nmax / (2.0L * c);
  const long double dw = theta ? 1.0L / kPiL : 2.0L / kPiL;  // dw / da
  for (int j = 0; j < nodes; ++j) {
    const long double a = kPiL * (long double)j / 1024.0L;
    const long double w = theta ? a / kPiL : 2.0L * a / kPiL - 1.0L;
    const long double th = tanhl(g * w);
    const long double sech2 = 1.0L - th * th;
    long double t = s * (th + c);
    if (j == 0) t = theta ? nmax / 2.0L : 0.0L;   // exact end points
    if (j == nodes - 1) t = theta ? nmax : nmax / 2.0L;
    const long double ti = floorl(t);
    const long double d1 = s * g * dw * sech2;
    const long double d2 = s * g * g * dw * dw * (-2.0L * sech2 * th) / 2.0L;
    out.push_back(TabEntry{(float)ti, (float)(t - ti), (float)d1, (float)d2});
  }
}

// cos, sin of pi k / M for k = 0 .. floor(M / 2): the per-code phi^ table of
// the fast decoders (exact values at k = 0 and 2k = M).
void phi_code_table(int M, std::vector<TabEntry> &out) {
  for (int k = 0; 2 * k <= M; ++k) {
    if (k == 0) {
      out.push_back(TabEntry{1.0f, 0.0f, 0.0f, 0.0f});
    } else if (2 * k == M) {
      out.push_back(TabEntry{0.0f, 0.0f, 1.0f, 0.0f});
    } else {
      const long double a = kPiL * (long double)k / (long double)M;
      out.push_back(entry_of(cosl(a), sinl(a)));
    }
  }
}

std::mutex g_mu;
std::map<TableKey, TableSet> g_tables;

ivc_status get_tables(const ivc_format *f, const Geometry &g, int device, TableSet *out) {
  TableKey key{device, f->map, g.N, g.M, f->map == IVC_MAP_TANH ? f->gamma : 0.0};
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_tables.find(key);
  if (it != g_tables.end()) {
    *out = it->second;
    return IVC_OK;
  }
  std::vector<TabEntry> host;
  TableSet ts;
  if (f->map == IVC_MAP_TANH) {
    const long double gm = (long double)f->gamma;
    ts.off_dec_t = host.size();
    for (int n = 0; n <= g.N; ++n) {
      long double psi = (n == 0) ? 0.0L : (n == g.N) ? 1.0L : (2LL * n == g.N) ? 0.5L
                        : psi_of_t((long double)n, (long double)g.N, gm);
      host.push_back(theta_entry_psi(psi));
    }
    ts.off_dec_p = host.size();
    for (int n = 0; n <= g.M; ++n) {
      long double psi = (n == 0) ? 0.0L : (n == g.M) ? 1.0L : (2LL * n == g.M) ? 0.5L
                        : psi_of_t((long double)n, (long double)g.M, gm);
      host.push_back(phi_entry_psi(psi));
    }
    ts.off_bnd_t = host.size();
    for (int k = 0; k < g.N; ++k) {
      long double psi = (2LL * k + 1 == g.N) ? 0.5L
                        : psi_of_t((long double)k + 0.5L, (long double)g.N, gm);
      host.push_back(theta_entry_psi(psi));
    }
    ts.off_bnd_p = host.size();
    for (int k = 0; k < g.M; ++k) {
      long double psi = (2LL * k + 1 == g.M) ? 0.5L
                        : psi_of_t((long double)k + 0.5L, (long double)g.M, gm);
      host.push_back(phi_entry_psi(psi));
    }
    ts.off_est = host.size();
    tanh_est_table((long double)g.N, gm, true, kTanhEstT, host);
    tanh_est_table((long double)g.M, gm, false, kTanhEstP, host);
  } else {
    uniform_table(g.N, host);
    ts.n_uniform_t = host.size();
    uniform_table(2 * g.M, host);
    ts.n_uniform_p = host.size() - ts.n_uniform_t;
    ts.off_phi = host.size();
    phi_code_table(g.M, host);
  }
  void *d = nullptr;
  if (cudaMalloc(&d, host.size() * sizeof(TabEntry)) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_NOMEM;
  }
  if (cudaMemcpy(d, host.data(), host.size() * sizeof(TabEntry), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    cudaFree(d);
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  ts.dev = static_cast<TabEntry *>(d);
  g_tables[key] = ts;
  *out = ts;
  return IVC_OK;
}

}  // namespace

void ivc::host_uniform_tables(const DevFormat &F, std::vector<TabEntry> &out) {
  uniform_table(F.Dt, out);
  uniform_table(F.Dp, out);
}

// Fills every field of *F except the table pointers (no device work).
ivc_status ivc::format_fields(const ivc_format *f, DevFormat *F, int *map_out) {
  Geometry g;
  ivc_status st = geometry(f, &g);
  if (st != IVC_OK) return st;
  std::memset(F, 0, sizeof(*F));
  F->sh_phi = (uint32_t)f->theta_bits;
  F->sh_m = (uint32_t)(f->theta_bits + f->phi_bits);
  F->sh_e = F->sh_m + (uint32_t)f->man_bits;
  F->mask_e = (1u << f->exp_bits) - 1u;
  F->mask_m = (1u << f->man_bits) - 1u;
  F->mask_phi = (1u << f->phi_bits) - 1u;
  F->mask_theta = (1u << f->theta_bits) - 1u;
  F->m_shift = (uint32_t)(23 - f->man_bits);
  const int P = f->phi_bits + f->theta_bits;
  F->mask_np = (P >= 64) ? ~0ull : ((1ull << P) - 1ull);
  F->e_off = f->exp_bias - 127;
  F->e_maxn = (1 << f->exp_bits) - 2;
  F->e_all = (1 << f->exp_bits) - 1;
  F->N = g.N;
  F->M = g.M;
  F->under_mode = f->underflow_mode;
  F->over_mode = f->overflow_mode;
  F->tscale_t = (float)((long double)g.N / (2.0L * kPiL));
  F->thalf_t = (float)(0.5L * g.N);
  F->tmax_t = (float)g.N - 0.25f;
  F->tscale_p = (float)((long double)g.M / kPiL);
  F->tmax_p = (float)g.M - 0.25f;
  F->Dt = g.N;
  F->Dp = 2 * g.M;
  F->st = table_shift(F->Dt);
  F->sp = table_shift(F->Dp);
  F->nent_t = table_entries(F->Dt, F->st);
  F->nent_p = table_entries(F->Dp, F->sp);
  ff_split(kPiL / (2.0L * F->Dt), F->Kt_h, F->Kt_l);
  ff_split(kPiL / (2.0L * F->Dp), F->Kp_h, F->Kp_l);
  exact::pi_over_host(2LL * F->Dt, F->Kxt_m, F->Kxt_e);
  exact::pi_over_host(2LL * F->Dp, F->Kxp_m, F->Kxp_e);
  F->tab = nullptr;
  {
    const unsigned __int128 two64 = (unsigned __int128)1 << 64;
    const unsigned __int128 d = (unsigned __int128)(g.N + 1);
    F->div_magic = (uint64_t)((two64 + d - 1) / d);
  }
  if (f->map == IVC_MAP_TANH) {
    F->gam = (float)f->gamma;
    F->tanh_c = (float)tanhl((long double)f->gamma);
    F->tanh_inv2c = (float)(1.0L / (2.0L * tanhl((long double)f->gamma)));
    F->nent_t = F->nent_p = 0;
    F->nest_t = kTanhEstT;
    F->nest_p = kTanhEstP;
  }
  *map_out = f->map;
  return IVC_OK;
}

namespace {

ivc_status make_devformat(const ivc_format *f, DevFormat *F, int *map_out) {
  ivc_status st = ivc::format_fields(f, F, map_out);
  if (st != IVC_OK) return st;
  Geometry g;
  geometry(f, &g);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  TableSet ts;
  st = get_tables(f, g, dev, &ts);
  if (st != IVC_OK) return st;
  F->tab = ts.dev;
  if (f->map != IVC_MAP_TANH) F->phi_tab = ts.dev + ts.off_phi;
  if (f->map == IVC_MAP_TANH) {
    F->dec_t = ts.dev + ts.off_dec_t;
    F->dec_p = ts.dev + ts.off_dec_p;
    F->bnd_t = ts.dev + ts.off_bnd_t;
    F->bnd_p = ts.dev + ts.off_bnd_p;
    F->est_tab = ts.dev + ts.off_est;
  }
  return IVC_OK;
}

// ------------------------------------------------------------ launch shapes

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

}  // namespace

LaunchShape ivc::default_shape(int map, int kind, const DevFormat &F, int64_t n, int vec2,
                               const ivc_launch_config *cfg) {
  LaunchShape s;
  s.block = (cfg && cfg->block > 0) ? cfg->block : 256;
  if (s.block > 256) s.block = 256;
  s.vec2 = vec2;
  s.smem = kernel_smem_bytes(F, map, kind, s.block);
  int bps = (cfg && cfg->blocks_per_sm > 0) ? cfg->blocks_per_sm : 0;
  const int occ = occupancy(map, kind, s.block, s.smem);
  if (bps <= 0 || (occ > 0 && bps > occ)) bps = occ > 0 ? occ : 1;
  const int64_t per_block = (int64_t)s.block * (vec2 ? 2 : 1);
  const int64_t need = (n + per_block - 1) / per_block;
  int64_t grid = (int64_t)sm_count() * bps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  s.grid = (int)grid;
  return s;
}

namespace {

ivc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return IVC_OK;
  return IVC_ERR_CUDA;
}

}  // namespace

// ===================================================================== ABI

extern "C" {

const char *ivc_status_string(ivc_status s) {
  switch (s) {
    case IVC_OK: return "ok";
    case IVC_ERR_ARG: return "invalid argument";
    case IVC_ERR_FORMAT: return "invalid or unsupported format";
    case IVC_ERR_ALIGN: return "misaligned pointer";
    case IVC_ERR_CUDA: return "CUDA runtime error";
    case IVC_ERR_TIMEOUT: return "bounded device loop ran out";
    case IVC_ERR_NOMEM: return "out of memory or workspace too small";
    case IVC_ERR_UNSUPPORTED: return "unsupported combination";
  }
  return "unknown status";
}

const char *ivc_version(void) { return "ivc 0.1 (sm_103a)"; }

ivc_status ivc_format_default(ivc_format *f) {
  if (!f) return IVC_ERR_ARG;
  std::memset(f, 0, sizeof(*f));
  f->sign_bits = 0;
  f->exp_bits = 7;
  f->man_bits = 22;
  f->phi_bits = 17;
  f->theta_bits = 18;
  f->exp_bias = 80;
  f->map = IVC_MAP_UNIFORM;
  f->gamma = 0.5;
  return IVC_OK;
}

ivc_status ivc_format_validate(const ivc_format *f) {
  Geometry g;
  return geometry(f, &g);
}

ivc_status ivc_release_tables(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_tables.begin(); it != g_tables.end();) {
    if (it->first.device == dev) {
      cudaFree(it->second.dev);
      it = g_tables.erase(it);
    } else {
      ++it;
    }
  }
  return IVC_OK;
}

ivc_status ivc_compress(const ivc_format *fmt, const float *xyz, ivc_layout layout, int64_t ld,
                        int64_t n, uint64_t *w, ivc_counts *counts, ivc_stream_t stream) {
  if (n < 0 || (layout != IVC_AOS && layout != IVC_SOA)) return IVC_ERR_ARG;
  if (layout == IVC_SOA && ld < n) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!xyz || !w) return IVC_ERR_ARG;
  if (!aligned(xyz, 4) || !aligned(w, 8) || (counts && !aligned(counts, 8))) return IVC_ERR_ALIGN;
  if (layout == IVC_AOS && aligned(xyz, 8) && aligned(w, 16) && fast::fast_geometry(map, F) != 0) {
    const LaunchShape s = default_shape(map, K_COMPRESS_FAST, F, n, 1, nullptr);
    return cuda_status(launch_compress_fast(F, xyz, n, w, counts, s, stream));
  }
  const LaunchShape s = default_shape(map, K_COMPRESS, F, n, 0, nullptr);
  return cuda_status(launch_compress(map, F, xyz, layout, ld, n, w, counts, s, stream));
}

ivc_status ivc_decompress(const ivc_format *fmt, const uint64_t *w, int64_t n, float *xyz,
                          ivc_layout layout, int64_t ld, ivc_stream_t stream) {
  if (n < 0 || (layout != IVC_AOS && layout != IVC_SOA)) return IVC_ERR_ARG;
  if (layout == IVC_SOA && ld < n) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!xyz || !w) return IVC_ERR_ARG;
  if (!aligned(xyz, 4) || !aligned(w, 8)) return IVC_ERR_ALIGN;
  if (layout == IVC_AOS && aligned(xyz, 8) && aligned(w, 16) && fast::fast_geometry(map, F) != 0) {
    const LaunchShape s = default_shape(map, K_DECOMPRESS_FAST, F, n, 1, nullptr);
    return cuda_status(launch_decompress_fast(F, w, n, xyz, s, stream));
  }
  const LaunchShape s = default_shape(map, K_DECOMPRESS, F, n, 0, nullptr);
  return cuda_status(launch_decompress(map, F, w, n, xyz, layout, ld, s, stream));
}

ivc_status ivc_compress_exact(const ivc_format *fmt, const float *xyz, int64_t n, uint64_t *w,
                              ivc_counts *counts, ivc_stream_t stream) {
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!xyz || !w) return IVC_ERR_ARG;
  if (!aligned(xyz, 4) || !aligned(w, 8) || (counts && !aligned(counts, 8))) return IVC_ERR_ALIGN;
  const LaunchShape s = default_shape(map, K_COMPRESS, F, n, 0, nullptr);
  return cuda_status(launch_compress_exact(map, F, xyz, n, w, counts, s, stream));
}

ivc_status ivc_decompress_exact(const ivc_format *fmt, const uint64_t *w, int64_t n, float *xyz,
                                ivc_stream_t stream) {
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!xyz || !w) return IVC_ERR_ARG;
  if (!aligned(xyz, 4) || !aligned(w, 8)) return IVC_ERR_ALIGN;
  const LaunchShape s = default_shape(map, K_DECOMPRESS, F, n, 0, nullptr);
  return cuda_status(launch_decompress_exact(map, F, w, n, xyz, s, stream));
}

ivc_status ivc_add_cfg(const ivc_format *fmt, const uint64_t *a, const uint64_t *b, uint64_t *c,
                       int64_t n, const ivc_launch_config *cfg, ivc_stream_t stream) {
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!a || !b || !c) return IVC_ERR_ARG;
  if (!aligned(a, 8) || !aligned(b, 8) || !aligned(c, 8)) return IVC_ERR_ALIGN;
  const int vec2 = (aligned(a, 16) && aligned(b, 16) && aligned(c, 16) &&
                    !(cfg && cfg->vec_per_thread == 1)) ? 1 : 0;
  if (vec2 && fast::fast_geometry(map, F) != 0) {
    const LaunchShape s = default_shape(map, K_ADD_FAST, F, n, 1, cfg);
    return cuda_status(launch_add_fast(F, a, b, c, n, s, stream));
  }
  const LaunchShape s = default_shape(map, K_ADD, F, n, vec2, cfg);
  return cuda_status(launch_add(map, F, a, b, c, n, s, stream));
}

ivc_status ivc_add(const ivc_format *fmt, const uint64_t *a, const uint64_t *b, uint64_t *c,
                   int64_t n, ivc_stream_t stream) {
  return ivc_add_cfg(fmt, a, b, c, n, nullptr, stream);
}

ivc_status ivc_axpy(const ivc_format *fmt, float alpha, const uint64_t *x, uint64_t *y, int64_t n,
                    ivc_stream_t stream) {
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!x || !y) return IVC_ERR_ARG;
  if (!aligned(x, 8) || !aligned(y, 8)) return IVC_ERR_ALIGN;
  const int vec2 = (aligned(x, 16) && aligned(y, 16)) ? 1 : 0;
  if (vec2 && fast::fast_geometry(map, F) != 0) {
    const LaunchShape s = default_shape(map, K_AXPY_FAST, F, n, 1, nullptr);
    return cuda_status(launch_axpy_fast(F, alpha, x, y, n, s, stream));
  }
  const LaunchShape s = default_shape(map, K_AXPY, F, n, vec2, nullptr);
  return cuda_status(launch_axpy(map, F, alpha, x, y, n, s, stream));
}

ivc_status ivc_pointwise_update(const ivc_format *fmt, float dt, const uint64_t *v,
                                const uint64_t *f, const float *rho, uint64_t *v_out,
                                uint64_t *m_out, int64_t n, ivc_stream_t stream) {
  if (n < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!v || !f || !v_out) return IVC_ERR_ARG;
  if (!aligned(v, 8) || !aligned(f, 8) || !aligned(v_out, 8) || (m_out && !aligned(m_out, 8)) ||
      (rho && !aligned(rho, 4)))
    return IVC_ERR_ALIGN;
  const bool al = aligned(v, 16) && aligned(f, 16) && aligned(v_out, 16) &&
                  (!m_out || aligned(m_out, 16)) && (!rho || aligned(rho, 8));
  if (al && fast::fast_geometry(map, F) != 0) {
    const LaunchShape s = default_shape(map, K_UPDATE_FAST, F, n, 1, nullptr);
    return cuda_status(launch_update_fast(F, dt, v, f, rho, v_out, m_out, n, s, stream));
  }
  const LaunchShape s = default_shape(map, K_UPDATE, F, n, 0, nullptr);
  return cuda_status(launch_update(map, F, dt, v, f, rho, v_out, m_out, n, s, stream));
}

// ------------------------------------------------------------------ gather

ivc_status ivc_gather_decompress(const ivc_format *fmt, const uint64_t *w, int64_t nw,
                                 const int64_t *idx, int64_t n, float *xyz,
                                 ivc_stream_t stream) {
  if (n < 0 || nw < 0) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = ivc::format_fields(fmt, &F, &map);
  if (st != IVC_OK) return st;
  if (n == 0) return IVC_OK;
  if (!idx || !xyz || (nw > 0 && !w)) return IVC_ERR_ARG;
  if ((w && !aligned(w, 8)) || !aligned(idx, 8) || !aligned(xyz, 4)) return IVC_ERR_ALIGN;
  st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  const bool pairs = aligned(idx, 16) && aligned(xyz, 8);
  return cuda_status(launch_gather(map, F, w, nw, idx, n, xyz, pairs, stream));
}

// ---------------------------------------------------------- flux divergence

namespace {

ivc_status fdiv_args(const void *F, int64_t ld, int ns, int nvars, int64_t ne, const float *D,
                     float *div, int64_t ld_out, size_t falign) {
  if (ne < 0 || ns < 1 || ns > 64 || nvars < 1 || nvars > 5) return IVC_ERR_ARG;
  if (ne == 0) return IVC_OK;
  if (ld < ne || ld_out < ne || !F || !D || !div) return IVC_ERR_ARG;
  if (!aligned(F, falign) || !aligned(D, 4) || !aligned(div, 4)) return IVC_ERR_ALIGN;
  return IVC_OK;
}

}  // namespace

namespace {

ivc_status flux_divergence(bool tc, const ivc_format *fmt, const uint64_t *F, int64_t ld, int ns,
                           int nvars, int64_t ne, const float *D, float *div, int64_t ld_out,
                           ivc_stream_t stream) {
  DevFormat Fm;
  int map;
  ivc_status st = ivc::format_fields(fmt, &Fm, &map);  // no device work yet
  if (st != IVC_OK) return st;
  st = fdiv_args(F, ld, ns, nvars, ne, D, div, ld_out, 8);
  if (st != IVC_OK || ne == 0) return st;
  st = make_devformat(fmt, &Fm, &map);
  if (st != IVC_OK) return st;
  const bool fastp = fast::fast_geometry(map, Fm) == 1;
  return cuda_status((tc ? launch_flux_div_tc : launch_flux_div)(map, fastp, false, Fm, F, ld, ns,
                                                                 nvars, ne, D, div, ld_out,
                                                                 stream));
}

ivc_status f32_flux_divergence(bool tc, const float *F, int64_t ld, int ns, int nvars, int64_t ne,
                               const float *D, float *div, int64_t ld_out, ivc_stream_t stream) {
  ivc_status st = fdiv_args(F, ld, ns, nvars, ne, D, div, ld_out, 4);
  if (st != IVC_OK || ne == 0) return st;
  DevFormat none{};
  return cuda_status((tc ? launch_flux_div_tc : launch_flux_div)(IVC_MAP_UNIFORM, false, true,
                                                                 none, F, ld, ns, nvars, ne, D,
                                                                 div, ld_out, stream));
}

}  // namespace

ivc_status ivc_flux_divergence(const ivc_format *fmt, const uint64_t *F, int64_t ld, int ns,
                               int nvars, int64_t ne, const float *D, float *div,
                               int64_t ld_out, ivc_stream_t stream) {
  return flux_divergence(true, fmt, F, ld, ns, nvars, ne, D, div, ld_out, stream);
}

ivc_status ivc_flux_divergence_simt(const ivc_format *fmt, const uint64_t *F, int64_t ld, int ns,
                                    int nvars, int64_t ne, const float *D, float *div,
                                    int64_t ld_out, ivc_stream_t stream) {
  return flux_divergence(false, fmt, F, ld, ns, nvars, ne, D, div, ld_out, stream);
}

ivc_status ivc_set_flux_divergence_wait_limit(long long cycles) {
  set_flux_div_wait_limit(cycles);
  return IVC_OK;
}

ivc_status ivc_flux_divergence_check(void) {
  int status = 0, status_tc = 0;
  if (flux_div_status(&status) != cudaSuccess || flux_div_tc_status(&status_tc) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  return (status || status_tc) ? IVC_ERR_TIMEOUT : IVC_OK;
}

ivc_status ivc_f32_flux_divergence(const float *F, int64_t ld, int ns, int nvars, int64_t ne,
                                   const float *D, float *div, int64_t ld_out,
                                   ivc_stream_t stream) {
  return f32_flux_divergence(true, F, ld, ns, nvars, ne, D, div, ld_out, stream);
}

ivc_status ivc_f32_flux_divergence_simt(const float *F, int64_t ld, int ns, int nvars, int64_t ne,
                                        const float *D, float *div, int64_t ld_out,
                                        ivc_stream_t stream) {
  return f32_flux_divergence(false, F, ld, ns, nvars, ne, D, div, ld_out, stream);
}

// ------------------------------------------------- flux reconstruction (5-11)

namespace {

// Validates the common arguments of an FR step and fills the call; `fmt`
// NULL selects FP32 rows.  Returns IVC_OK with call->ne == 0 for empty work.
ivc_status fr_prepare(int step, const ivc_format *fmt, const ivc_fr_basis *basis, int order,
                      const ivc_fr_gas *gas, int64_t ne, int64_t ld, int nvars,
                      std::initializer_list<const void *> ins, void *out, FrCall *call) {
  *call = FrCall{};
  call->step = step;
  call->f32 = fmt == nullptr;
  if (fmt) {
    ivc_status st = ivc::format_fields(fmt, &call->F, &call->map);
    if (st != IVC_OK) return st;
  }
  if (basis) {
    call->basis = *basis;
    order = basis->order;
  } else {
    call->basis.order = order;
  }
  if (order < 1 || order > 3 || nvars < 1 || nvars > 5 || ne < 0) return IVC_ERR_ARG;
  if (gas) call->gas = *gas;
  call->ne = ne;
  call->ld = ld;
  call->nv = nvars;
  if (ne == 0) return IVC_OK;
  if (ld < ne || !out) return IVC_ERR_ARG;
  const void *p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int i = 0;
  for (const void *x : ins) {
    if (!x) return IVC_ERR_ARG;
    if (!aligned(x, 4)) return IVC_ERR_ALIGN;
    p[i++] = x;
  }
  if (!aligned(out, 4)) return IVC_ERR_ALIGN;
  call->in0 = p[0];
  call->in1 = p[1];
  call->in2 = p[2];
  call->in3 = p[3];
  call->in4 = p[4];
  call->in5 = p[5];
  call->out = out;
  return IVC_OK;
}

// Word arrays must be 8-byte aligned.
ivc_status words_aligned(std::initializer_list<const void *> ws) {
  for (const void *w : ws)
    if (w && !aligned(w, 8)) return IVC_ERR_ALIGN;
  return IVC_OK;
}

ivc_status fr_run(FrCall &call, const ivc_format *fmt, ivc_stream_t stream) {
  if (call.ne == 0) return IVC_OK;
  if (fmt) {
    ivc_status st = make_devformat(fmt, &call.F, &call.map);
    if (st != IVC_OK) return st;
  }
  return cuda_status(launch_fr(call, stream));
}

}  // namespace

ivc_status ivc_fr_gradient(const ivc_format *fmt, const ivc_fr_basis *basis, const float *w,
                           int64_t ne, int64_t ld, int nvars, uint64_t *grad,
                           ivc_stream_t stream) {
  if (!fmt || !basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(5, fmt, basis, 0, nullptr, ne, ld, nvars, {w}, grad, &c);
  if (st == IVC_OK && ne > 0) st = words_aligned({grad});
  return st != IVC_OK ? st : fr_run(c, fmt, stream);
}

ivc_status ivc_f32_fr_gradient(const ivc_fr_basis *basis, const float *w, int64_t ne,
                               int64_t ld, int nvars, float *grad, ivc_stream_t stream) {
  if (!basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(5, nullptr, basis, 0, nullptr, ne, ld, nvars, {w}, grad, &c);
  return st != IVC_OK ? st : fr_run(c, nullptr, stream);
}

ivc_status ivc_fr_correct_gradient(const ivc_format *fmt, const ivc_fr_basis *basis,
                                   const uint64_t *grad, const float *dw, int64_t ne, int64_t ld,
                                   int nvars, uint64_t *grad_c, ivc_stream_t stream) {
  if (!fmt || !basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(6, fmt, basis, 0, nullptr, ne, ld, nvars, {grad, dw}, grad_c, &c);
  if (st == IVC_OK && ne > 0) st = words_aligned({grad, grad_c});
  return st != IVC_OK ? st : fr_run(c, fmt, stream);
}

ivc_status ivc_f32_fr_correct_gradient(const ivc_fr_basis *basis, const float *grad,
                                       const float *dw, int64_t ne, int64_t ld, int nvars,
                                       float *grad_c, ivc_stream_t stream) {
  if (!basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(6, nullptr, basis, 0, nullptr, ne, ld, nvars, {grad, dw}, grad_c,
                             &c);
  return st != IVC_OK ? st : fr_run(c, nullptr, stream);
}

ivc_status ivc_fr_interp_rows(const ivc_format *fmt, const ivc_fr_basis *basis,
                              const uint64_t *rows, int64_t ne, int64_t ld, int nvars,
                              uint64_t *rows_f, ivc_stream_t stream) {
  if (!fmt || !basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(7, fmt, basis, 0, nullptr, ne, ld, nvars, {rows}, rows_f, &c);
  if (st == IVC_OK && ne > 0) st = words_aligned({rows, rows_f});
  return st != IVC_OK ? st : fr_run(c, fmt, stream);
}

ivc_status ivc_f32_fr_interp_rows(const ivc_fr_basis *basis, const float *rows, int64_t ne,
                                  int64_t ld, int nvars, float *rows_f, ivc_stream_t stream) {
  if (!basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(7, nullptr, basis, 0, nullptr, ne, ld, nvars, {rows}, rows_f, &c);
  return st != IVC_OK ? st : fr_run(c, nullptr, stream);
}

namespace {

ivc_status fr_common_viscous(const ivc_format *fmt, int order, const ivc_fr_gas *gas,
                             const int dims[3], const void *grad_f, const void *nrm,
                             const void *S_f, const float *detJ_f, const float *q_f,
                             const float *nFinv, int64_t ld, float *out, ivc_stream_t stream) {
  if (!gas || !dims) return IVC_ERR_ARG;
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return IVC_ERR_ARG;
  const int64_t ne = (int64_t)dims[0] * dims[1] * dims[2];
  FrCall c;
  ivc_status st = fr_prepare(8, fmt, nullptr, order, gas, ne, ld, 5,
                             {grad_f, nrm, S_f, detJ_f, q_f, nFinv}, out, &c);
  if (st == IVC_OK && fmt) st = words_aligned({grad_f, nrm, S_f});
  if (st != IVC_OK) return st;
  for (int i = 0; i < 3; ++i) c.dims[i] = dims[i];
  return fr_run(c, fmt, stream);
}

}  // namespace

ivc_status ivc_fr_common_viscous_flux(const ivc_format *fmt, int order, const ivc_fr_gas *gas,
                                      const int dims[3], const uint64_t *grad_f,
                                      const uint64_t *nrm, const uint64_t *S_f,
                                      const float *detJ_f, const float *q_f, const float *nFinv,
                                      int64_t ld, float *out, ivc_stream_t stream) {
  if (!fmt) return IVC_ERR_ARG;
  return fr_common_viscous(fmt, order, gas, dims, grad_f, nrm, S_f, detJ_f, q_f, nFinv, ld, out,
                           stream);
}

ivc_status ivc_f32_fr_common_viscous_flux(int order, const ivc_fr_gas *gas, const int dims[3],
                                          const float *grad_f, const float *nrm,
                                          const float *S_f, const float *detJ_f,
                                          const float *q_f, const float *nFinv, int64_t ld,
                                          float *out, ivc_stream_t stream) {
  return fr_common_viscous(nullptr, order, gas, dims, grad_f, nrm, S_f, detJ_f, q_f, nFinv, ld,
                           out, stream);
}

ivc_status ivc_fr_flux(const ivc_format *fmt, int order, const ivc_fr_gas *gas, const float *q_s,
                       const uint64_t *grad, const uint64_t *S_s, const float *detJ_s,
                       int64_t ne, int64_t ld, uint64_t *F, ivc_stream_t stream) {
  if (!fmt || !gas) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(9, fmt, nullptr, order, gas, ne, ld, 5, {q_s, grad, S_s, detJ_s}, F,
                             &c);
  if (st == IVC_OK && ne > 0) st = words_aligned({grad, S_s, F});
  return st != IVC_OK ? st : fr_run(c, fmt, stream);
}

ivc_status ivc_f32_fr_flux(int order, const ivc_fr_gas *gas, const float *q_s, const float *grad,
                           const float *S_s, const float *detJ_s, int64_t ne, int64_t ld,
                           float *F, ivc_stream_t stream) {
  if (!gas) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(9, nullptr, nullptr, order, gas, ne, ld, 5,
                             {q_s, grad, S_s, detJ_s}, F, &c);
  return st != IVC_OK ? st : fr_run(c, nullptr, stream);
}

ivc_status ivc_fr_flux_correction(const ivc_format *fmt, const ivc_fr_basis *basis,
                                  const uint64_t *F, const float *nF, int64_t ne, int64_t ld,
                                  int nvars, float *Fc, ivc_stream_t stream) {
  if (!fmt || !basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(11, fmt, basis, 0, nullptr, ne, ld, nvars, {F, nF}, Fc, &c);
  if (st == IVC_OK && ne > 0) st = words_aligned({F});
  return st != IVC_OK ? st : fr_run(c, fmt, stream);
}

ivc_status ivc_f32_fr_flux_correction(const ivc_fr_basis *basis, const float *F, const float *nF,
                                      int64_t ne, int64_t ld, int nvars, float *Fc,
                                      ivc_stream_t stream) {
  if (!basis) return IVC_ERR_ARG;
  FrCall c;
  ivc_status st = fr_prepare(11, nullptr, basis, 0, nullptr, ne, ld, nvars, {F, nF}, Fc, &c);
  return st != IVC_OK ? st : fr_run(c, nullptr, stream);
}

// ------------------------------------------------------------------ batched

struct ivc_plan_s {
  int device = 0;
  int map = 0;
  int op = 0;
  DevFormat F{};
  PlanDev P{};
  LaunchShape shape{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static size_t plan_ws_bytes(int nfields) {
  size_t b = round_up(sizeof(FieldDesc) * (size_t)nfields, 256);
  b += round_up(sizeof(int64_t) * (size_t)(nfields + 1), 256);
  b += 256;  // counter + status
  return b;
}

ivc_status ivc_plan_batched(const ivc_format *fmt, ivc_op op, const ivc_field *fields,
                            int nfields, void *workspace, size_t *ws_bytes,
                            const ivc_launch_config *cfg, ivc_stream_t stream, ivc_plan *plan) {
  if (!ws_bytes || nfields < 1 || (op != IVC_OP_ADD && op != IVC_OP_AXPY)) return IVC_ERR_ARG;
  const size_t need = plan_ws_bytes(nfields);
  if (!workspace) {
    *ws_bytes = need;
    return IVC_OK;
  }
  if (!fields || !plan) return IVC_ERR_ARG;
  if (*ws_bytes < need) return IVC_ERR_NOMEM;
  if (!aligned(workspace, 256)) return IVC_ERR_ALIGN;
  int64_t total_n = 0;
  for (int i = 0; i < nfields; ++i) {
    const ivc_field &f = fields[i];
    if (f.n < 0) return IVC_ERR_ARG;
    if (f.n > 0 && (!f.a || !f.c || (op == IVC_OP_ADD && !f.b))) return IVC_ERR_ARG;
    if (!aligned(f.a, 8) || !aligned(f.c, 8) || (f.b && !aligned(f.b, 8))) return IVC_ERR_ALIGN;
    total_n += f.n;
  }
  ivc_plan_s *p = new ivc_plan_s();
  ivc_status st = make_devformat(fmt, &p->F, &p->map);
  if (st != IVC_OK) {
    delete p;
    return st;
  }
  p->op = op;
  cudaGetDevice(&p->device);
  int tile = (cfg && cfg->tile > 0) ? cfg->tile : 8192;
  tile = (tile + 1) & ~1;  // even tiles keep 16-byte alignment inside a field
  char *ws = static_cast<char *>(workspace);
  FieldDesc *d_fields = reinterpret_cast<FieldDesc *>(ws);
  ws += round_up(sizeof(FieldDesc) * (size_t)nfields, 256);
  int64_t *d_tiles = reinterpret_cast<int64_t *>(ws);
  ws += round_up(sizeof(int64_t) * (size_t)(nfields + 1), 256);
  unsigned long long *d_counter = reinterpret_cast<unsigned long long *>(ws);
  int *d_status = reinterpret_cast<int *>(ws + 64);

  std::vector<FieldDesc> h(nfields);
  int64_t total_tiles = 0;
  for (int i = 0; i < nfields; ++i) {
    h[i] = FieldDesc{fields[i].a, op == IVC_OP_ADD ? fields[i].b : nullptr, fields[i].c,
                     fields[i].n, fields[i].alpha, 0.0f};
    total_tiles += (fields[i].n + tile - 1) / tile;
  }
  cudaError_t e = cudaMemcpyAsync(d_fields, h.data(), sizeof(FieldDesc) * nfields,
                                  cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = launch_tile_scan(d_fields, nfields, tile, d_tiles, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int), stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host copy source must outlive it
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return IVC_ERR_CUDA;
  }
  p->P = PlanDev{d_fields, d_tiles, d_counter, d_status, total_tiles, nfields, tile};
  const bool fastp = fast::fast_geometry(p->map, p->F) != 0;
  const int kind = op == IVC_OP_ADD ? (fastp ? K_BATCH_ADD_FAST : K_BATCH_ADD)
                                    : (fastp ? K_BATCH_AXPY_FAST : K_BATCH_AXPY);
  LaunchShape s;
  s.block = (cfg && cfg->block > 0 && cfg->block <= 256) ? cfg->block : 256;
  s.vec2 = 1;
  s.smem = kernel_smem_bytes(p->F, p->map, kind, s.block);
  const int occ = occupancy(p->map, kind, s.block, s.smem);
  int bps = (cfg && cfg->blocks_per_sm > 0) ? cfg->blocks_per_sm : occ;
  if (occ > 0 && bps > occ) bps = occ;
  if (bps < 1) bps = 1;
  int64_t grid = (int64_t)sm_count() * bps;
  if (grid > total_tiles) grid = total_tiles > 0 ? total_tiles : 1;
  s.grid = (int)grid;
  p->shape = s;
  (void)total_n;

  // Capture counter reset + persistent launch into a graph on a private stream.
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), cap);
    cudaError_t e2 = e1 == cudaSuccess ? launch_batched(p->map, op, p->F, p->P, s, cap) : e1;
    cudaError_t e3 = cudaStreamEndCapture(cap, &p->graph);
    e = e2 != cudaSuccess ? e2 : e3;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
    return IVC_ERR_CUDA;
  }
  *plan = p;
  return IVC_OK;
}

ivc_status ivc_launch_plan(ivc_plan plan, ivc_stream_t stream) {
  if (!plan || !plan->exec) return IVC_ERR_ARG;
  return cuda_status(cudaGraphLaunch(plan->exec, stream));
}

ivc_status ivc_launch_plan_direct(ivc_plan plan, ivc_stream_t stream) {
  if (!plan) return IVC_ERR_ARG;
  cudaError_t e = cudaMemsetAsync(plan->P.counter, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) e = launch_batched(plan->map, plan->op, plan->F, plan->P, plan->shape, stream);
  return cuda_status(e);
}

ivc_status ivc_plan_status(ivc_plan plan, ivc_stream_t stream) {
  if (!plan) return IVC_ERR_ARG;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, plan->P.status, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return IVC_ERR_CUDA;
  return (ivc_status)h;
}

ivc_status ivc_plan_destroy(ivc_plan plan) {
  if (!plan) return IVC_ERR_ARG;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
  return IVC_OK;
}

// ------------------------------------------------------------------ tuner

ivc_status ivc_tune_batched(const ivc_format *fmt, ivc_op op, const ivc_field *fields,
                            int nfields, void *workspace, size_t ws_bytes, ivc_stream_t stream,
                            ivc_launch_config *best) {
  if (!best || !fields || nfields < 1 || !workspace) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  const bool fastp = fast::fast_geometry(map, F) != 0;
  const int kind = op == IVC_OP_ADD ? (fastp ? K_BATCH_ADD_FAST : K_BATCH_ADD)
                                    : (fastp ? K_BATCH_AXPY_FAST : K_BATCH_AXPY);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  const int blocks[] = {128, 256};
  const int tiles[] = {2048, 8192, 32768, 131072};
  float best_ms = 1e30f;
  ivc_launch_config bc{256, fastp ? 2 : 1, 8192, 0};
  ivc_status err = IVC_OK;
  for (int blk : blocks) {
    const int occ = occupancy(map, kind, blk, kernel_smem_bytes(F, map, kind, blk));
    for (int bps = 1; bps <= occ && err == IVC_OK; bps = (bps * 2 > occ && bps < occ) ? occ : bps * 2) {
      for (int tile : tiles) {
        const ivc_launch_config cfg{blk, fastp ? 2 : 1, tile, bps};
        size_t ws = ws_bytes;
        ivc_plan plan = nullptr;
        err = ivc_plan_batched(fmt, op, fields, nfields, workspace, &ws, &cfg, stream, &plan);
        if (err != IVC_OK) break;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3 && err == IVC_OK; ++rep) {
          cudaEventRecord(e0, stream);
          err = ivc_launch_plan_direct(plan, stream);
          cudaEventRecord(e1, stream);
          if (err == IVC_OK && cudaEventSynchronize(e1) != cudaSuccess) err = IVC_ERR_CUDA;
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0 && ms < ms_min) ms_min = ms;
        }
        const ivc_status ps = err == IVC_OK ? ivc_plan_status(plan, stream) : err;
        ivc_plan_destroy(plan);
        if (err == IVC_OK) err = ps;
        if (err != IVC_OK) break;
        if (ms_min < best_ms) {
          best_ms = ms_min;
          bc = cfg;
        }
      }
    }
    if (err != IVC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != IVC_OK) {
    cudaGetLastError();
    return err;
  }
  *best = bc;
  return IVC_OK;
}

ivc_status ivc_tune(const ivc_format *fmt, ivc_op op, const uint64_t *a, const uint64_t *b,
                    uint64_t *c, int64_t n, ivc_stream_t stream, ivc_launch_config *best) {
  if (!best || n <= 0 || !a || !b || (op == IVC_OP_ADD && !c)) return IVC_ERR_ARG;
  DevFormat F;
  int map;
  ivc_status st = make_devformat(fmt, &F, &map);
  if (st != IVC_OK) return st;
  const int kind = op == IVC_OP_ADD ? K_ADD : K_AXPY;
  const int vec2 = (aligned(a, 16) && aligned(b, 16) && (!c || aligned(c, 16))) ? 1 : 0;
  const int blocks[] = {64, 128, 256};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return IVC_ERR_CUDA;
  }
  float best_ms = 1e30f;
  ivc_launch_config bc{256, vec2 ? 2 : 1, 8192, 0};
  const bool fast_kind = vec2 && fast::fast_geometry(map, F) != 0;
  for (int blk : blocks) {
    const int okind = fast_kind ? (op == IVC_OP_ADD ? K_ADD_FAST : K_AXPY_FAST) : kind;
    const size_t smem = kernel_smem_bytes(F, map, okind, blk);
    const int occ = occupancy(map, okind, blk, smem);
    for (int bps = 1; bps <= occ; bps *= 2) {
      ivc_launch_config cfg{blk, vec2 ? 2 : 1, 8192, bps};
      LaunchShape s = default_shape(map, kind, F, n, vec2, &cfg);
      float ms_min = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, stream);
        const bool fastp = vec2 && fast::fast_geometry(map, F) != 0;
        cudaError_t e;
        if (fastp) {
          const LaunchShape sf =
              default_shape(map, op == IVC_OP_ADD ? K_ADD_FAST : K_AXPY_FAST, F, n, 1, &cfg);
          e = op == IVC_OP_ADD
                  ? launch_add_fast(F, a, b, c, n, sf, stream)
                  : launch_axpy_fast(F, 0.7f, a, const_cast<uint64_t *>(b), n, sf, stream);
        } else {
          e = op == IVC_OP_ADD ? launch_add(map, F, a, b, c, n, s, stream)
                               : launch_axpy(map, F, 0.7f, a, const_cast<uint64_t *>(b), n, s,
                                             stream);
        }
        cudaEventRecord(e1, stream);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          cudaGetLastError();
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return IVC_ERR_CUDA;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < ms_min) ms_min = ms;
      }
      if (ms_min < best_ms) {
        best_ms = ms_min;
        bc = cfg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best = bc;
  return IVC_OK;
}

}  // extern "C"
