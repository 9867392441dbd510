// api.cu -- host side of the C ABI declared in include/gpet.h: scanner
// descriptions (Sec. 2.1 hierarchy; repetition mode or panels placed one by
// one), phantom upload and validation, the cross-section table, errors.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "gpet.h"
#include "internal.h"
#include "host.h"

using namespace gpet;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_err = "no error";

int gpet_fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int gpet_cuda_fail(cudaError_t e, const char *where) {
    return gpet_fail(GPET_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" const char *gpet_last_error(void) { return t_err.c_str(); }
extern "C" const char *gpet_version(void) { return "gpet-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// kernel loading and shared-memory limits (see internal.h)
// ---------------------------------------------------------------------------
namespace gpet {

static std::mutex g_attr_mutex;
static std::map<std::pair<int, const void *>, size_t> g_smem_limit;  // (device, kernel) -> limit set

cudaError_t ensure_dynamic_smem(const void *fn, size_t bytes) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // the limit covers the kernel's static shared memory as well
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const size_t cap = optin > (int)fa.sharedSizeBytes ? (size_t)(optin - (int)fa.sharedSizeBytes) : 0;
    bytes = std::min(bytes, cap);
    std::lock_guard<std::mutex> lk(g_attr_mutex);
    size_t &have = g_smem_limit[std::make_pair(dev, fn)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

cudaError_t preload_kernels() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    e = preload_transport_kernels();
    if (e == cudaSuccess) e = preload_sort_kernels();
    if (e == cudaSuccess) e = preload_window_kernels();
    if (e == cudaSuccess) e = preload_copy_kernels();
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

}  // namespace gpet

// ---------------------------------------------------------------------------
// Klein-Nishina ratio table g(E) = sigma_KN(E) / sigma_KN(511 keV), built in
// FP64 on the host, stored FP32 on a log-E grid from 1 keV to 511 keV
// ---------------------------------------------------------------------------
static double kn_total(double e_kev) {
    const double k = e_kev / 510.99895;
    const double a = 1.0 + 2.0 * k;
    const double l = std::log(a);
    // 2 pi r_e^2 factor omitted: only ratios are used
    return (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k) + l / (2.0 * k) - (1.0 + 3.0 * k) / (a * a);
}

static std::mutex g_tab_mutex;
static float *g_tab_dev[64] = {nullptr};

int gpet_xs_table(const float **out, float *ln_emin, float *inv_h) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return gpet_fail(GPET_ERR_INVALID_ARG, "device index %d out of range", dev);
    const double lmin = std::log((double)kXsEmin), lmax = std::log(511.0);
    const double h = (lmax - lmin) / kXsIntervals;
    *ln_emin = (float)lmin;
    *inv_h = (float)(1.0 / h);
    std::lock_guard<std::mutex> lk(g_tab_mutex);
    if (!g_tab_dev[dev]) {
        std::vector<float> t(kXsIntervals + 1);
        const double s511 = kn_total(511.0);
        for (int i = 0; i <= kXsIntervals; ++i) {
            const double E = i == kXsIntervals ? 511.0 : std::exp(lmin + h * i);
            t[i] = (float)(kn_total(E) / s511);
        }
        t[kXsIntervals] = 1.0f;
        float *d = nullptr;
        e = cudaMalloc(&d, sizeof(float) * t.size());
        if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaMalloc(xs table)");
        e = cudaMemcpy(d, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(d); return gpet_cuda_fail(e, "cudaMemcpy(xs table)"); }
        g_tab_dev[dev] = d;
    }
    *out = g_tab_dev[dev];
    return GPET_OK;
}

// ---------------------------------------------------------------------------
// scanner
// ---------------------------------------------------------------------------
static double mu_c511(const gpet_material &m) {
    if (m.electron_density_cm3 > 0.0) {
        const double re = 2.8179403262e-13;
        return m.electron_density_cm3 * 2.0 * M_PI * re * re * kn_total(511.0);
    }
    return m.mu_total_511_cm * (1.0 - m.photo_frac_511);
}

static bool material_ok(const gpet_material &m) {
    return std::isfinite(m.mu_total_511_cm) && m.mu_total_511_cm >= 0.0 && m.photo_frac_511 >= 0.0 &&
           m.photo_frac_511 <= 1.0 && std::isfinite(m.electron_density_cm3) && m.electron_density_cm3 >= 0.0;
}

// separating-axis test of two panel boxes projected on the transaxial plane
static bool panels_overlap(double R, double W, double half_u, double a0, double a1) {
    auto corners = [&](double a, double pts[4][2]) {
        const double c = std::cos(a), s = std::sin(a);
        const double ws[2] = {R, R + W}, us[2] = {-half_u, half_u};
        int q = 0;
        for (double w : ws)
            for (double u : us) { pts[q][0] = w * c - u * s; pts[q][1] = w * s + u * c; ++q; }
    };
    double p0[4][2], p1[4][2];
    corners(a0, p0);
    corners(a1, p1);
    const double axes[4][2] = {{std::cos(a0), std::sin(a0)}, {-std::sin(a0), std::cos(a0)},
                               {std::cos(a1), std::sin(a1)}, {-std::sin(a1), std::cos(a1)}};
    const double eps = 1e-9 * (R + W + half_u);
    for (auto &ax : axes) {
        double lo0 = 1e300, hi0 = -1e300, lo1 = 1e300, hi1 = -1e300;
        for (int q = 0; q < 4; ++q) {
            const double v0 = p0[q][0] * ax[0] + p0[q][1] * ax[1];
            const double v1 = p1[q][0] * ax[0] + p1[q][1] * ax[1];
            lo0 = std::min(lo0, v0); hi0 = std::max(hi0, v0);
            lo1 = std::min(lo1, v1); hi1 = std::max(hi1, v1);
        }
        if (hi0 <= lo1 + eps || hi1 <= lo0 + eps) return false;  // separated (touching allowed)
    }
    return true;
}

// oriented box of posed panel k: centre, axes (rows w, u, v) and half extents
struct Obb {
    double c[3], a[3][3], e[3];
};

static Obb posed_box(const double *P, double W, double U, double V) {
    Obb b;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b.a[i][j] = P[3 * i + j];
    for (int j = 0; j < 3; ++j) b.c[j] = P[9 + j] + 0.5 * W * P[j];
    b.e[0] = 0.5 * W; b.e[1] = 0.5 * U; b.e[2] = 0.5 * V;
    return b;
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// separating-axis test of two oriented boxes (face normals of both and their
// nine cross products); touching boxes do not overlap
static bool boxes_overlap(const Obb &A, const Obb &B) {
    double axes[15][3];
    int n = 0;
    for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) axes[n][j] = A.a[i][j]; ++n; }
    for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) axes[n][j] = B.a[i][j]; ++n; }
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            const double *p = A.a[i], *q = B.a[k];
            double x[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]};
            const double nn = std::sqrt(dot3(x, x));
            if (nn < 1e-9) continue;  // parallel edges: covered by the face normals
            for (int j = 0; j < 3; ++j) axes[n][j] = x[j] / nn;
            ++n;
        }
    const double scale = std::max({A.e[0], A.e[1], A.e[2], B.e[0], B.e[1], B.e[2], 1.0});
    for (int t = 0; t < n; ++t) {
        const double *L = axes[t];
        double ra = 0.0, rb = 0.0;
        for (int i = 0; i < 3; ++i) {
            ra += A.e[i] * std::fabs(dot3(A.a[i], L));
            rb += B.e[i] * std::fabs(dot3(B.a[i], L));
        }
        const double d[3] = {B.c[0] - A.c[0], B.c[1] - A.c[1], B.c[2] - A.c[2]};
        if (std::fabs(dot3(d, L)) >= ra + rb - 1e-9 * scale) return false;  // separated (touching allowed)
    }
    return true;
}

// non-repetition mode: validate the poses, reject overlapping panels and
// build the device table (4 float4 per panel: axis + axis.origin, then origin)
static int build_poses(const gpet_scanner_desc *d, double W, double U, double V, std::vector<float> &out) {
    const double *P = d->panel_poses;
    for (int k = 0; k < d->n_panels; ++k) {
        const double *p = P + 12 * k;
        for (int j = 0; j < 12; ++j)
            if (!std::isfinite(p[j])) return gpet_fail(GPET_ERR_INVALID_ARG, "panel %d: pose entry %d not finite", k, j);
        for (int i = 0; i < 3; ++i)
            if (std::fabs(dot3(p + 3 * i, p + 3 * i) - 1.0) > 2e-6)
                return gpet_fail(GPET_ERR_GEOMETRY, "panel %d: pose axis %d is not a unit vector", k, i);
        if (std::fabs(dot3(p, p + 3)) > 1e-6 || std::fabs(dot3(p, p + 6)) > 1e-6 || std::fabs(dot3(p + 3, p + 6)) > 1e-6)
            return gpet_fail(GPET_ERR_GEOMETRY, "panel %d: pose axes are not orthogonal", k);
        const double cx[3] = {p[1] * p[5] - p[2] * p[4], p[2] * p[3] - p[0] * p[5], p[0] * p[4] - p[1] * p[3]};
        if (dot3(cx, p + 6) < 1.0 - 1e-6)
            return gpet_fail(GPET_ERR_GEOMETRY, "panel %d: pose axes are not right-handed (v != w x u)", k);
    }
    for (int a = 0; a < d->n_panels; ++a)
        for (int b = a + 1; b < d->n_panels; ++b)
            if (boxes_overlap(posed_box(P + 12 * a, W, U, V), posed_box(P + 12 * b, W, U, V)))
                return gpet_fail(GPET_ERR_GEOMETRY, "posed panels %d and %d overlap", a, b);
    out.assign((size_t)16 * d->n_panels, 0.0f);
    for (int k = 0; k < d->n_panels; ++k) {
        const double *p = P + 12 * k;
        float *q = out.data() + 16 * k;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) q[4 * i + j] = (float)p[3 * i + j];
            q[4 * i + 3] = (float)dot3(p + 3 * i, p + 9);
        }
        for (int j = 0; j < 3; ++j) q[12 + j] = (float)p[9 + j];
    }
    return GPET_OK;
}

int gpet_build_geometry(const gpet_scanner_desc *d, GeomDev &g, int64_t &n_crystals, std::vector<float> *pose_dev) {
    if (!d) return gpet_fail(GPET_ERR_INVALID_ARG, "scanner description is NULL");
    if (d->n_panels < 1 || d->n_panels > kMaxPanels)
        return gpet_fail(GPET_ERR_INVALID_ARG, "n_panels=%d outside [1, %d]", d->n_panels, kMaxPanels);
    if (d->n_layers < 1 || d->n_layers > kMaxLayers || !d->layers)
        return gpet_fail(GPET_ERR_INVALID_ARG, "n_layers=%d outside [1, %d] or layers NULL", d->n_layers, kMaxLayers);
    if (d->n_materials < 1 || d->n_materials > kMaxMaterials || !d->materials)
        return gpet_fail(GPET_ERR_INVALID_ARG, "n_materials=%d outside [1, %d] or materials NULL", d->n_materials,
                         kMaxMaterials);
    if (d->modules_u < 1 || d->modules_v < 1)
        return gpet_fail(GPET_ERR_INVALID_ARG, "modules %d x %d", d->modules_u, d->modules_v);
    const bool posed = d->panel_poses != nullptr;
    if (!(posed || d->inner_radius_mm > 0.0) || !(d->module_size_u > 0.0) || !(d->module_size_v > 0.0) ||
        !(d->module_gap_u >= 0.0) || !(d->module_gap_v >= 0.0) || !std::isfinite(d->first_angle_rad))
        return gpet_fail(GPET_ERR_GEOMETRY, "radius, module sizes must be > 0 and module gaps >= 0");
    if (d->readout_level != 0 && d->readout_level != 1 && d->readout_level != 3)
        return gpet_fail(GPET_ERR_INVALID_ARG, "readout_level %d not in {0, 1, 3}", d->readout_level);
    for (int m = 0; m < d->n_materials; ++m)
        if (!material_ok(d->materials[m])) return gpet_fail(GPET_ERR_INVALID_ARG, "material %d out of range", m);
    std::memset(&g, 0, sizeof(g));
    g.n_panels = d->n_panels;
    g.n_layers = d->n_layers;
    g.n_materials = d->n_materials;
    g.modules_u = d->modules_u;
    g.modules_v = d->modules_v;
    g.readout_level = d->readout_level;
    const double U = d->modules_u * d->module_size_u + (d->modules_u - 1) * d->module_gap_u;
    const double V = d->modules_v * d->module_size_v + (d->modules_v - 1) * d->module_gap_v;
    double w = 0.0;
    int32_t loff = 0;
    for (int l = 0; l < d->n_layers; ++l) {
        const gpet_layer &L = d->layers[l];
        if (L.n_u < 1 || L.n_v < 1) return gpet_fail(GPET_ERR_GEOMETRY, "layer %d has %d x %d crystals", l, L.n_u, L.n_v);
        if (!(L.pitch_u > 0.0) || !(L.pitch_v > 0.0) || !(L.gap_u >= 0.0) || !(L.gap_v >= 0.0) ||
            !(L.gap_u < L.pitch_u) || !(L.gap_v < L.pitch_v))
            return gpet_fail(GPET_ERR_GEOMETRY, "layer %d: need pitch > gap >= 0", l);
        if (!(L.depth > 0.0) || !(L.gap_before >= 0.0) || !(L.offset_u >= 0.0) || !(L.offset_v >= 0.0))
            return gpet_fail(GPET_ERR_GEOMETRY, "layer %d: need depth > 0, gap_before >= 0, offsets >= 0", l);
        const double tol = 1e-9;
        if (L.offset_u + L.n_u * L.pitch_u > d->module_size_u * (1 + tol) + tol ||
            L.offset_v + L.n_v * L.pitch_v > d->module_size_v * (1 + tol) + tol)
            return gpet_fail(GPET_ERR_GEOMETRY, "layer %d: crystal grid leaves its module", l);
        if (L.crystal_mat < 0 || L.crystal_mat >= d->n_materials || L.interval_mat < 0 ||
            L.interval_mat >= d->n_materials)
            return gpet_fail(GPET_ERR_INVALID_ARG, "layer %d: material index out of range", l);
        LayerDev &Ld = g.layers[l];
        w += L.gap_before;
        Ld.w0 = (float)w;
        w += L.depth;
        Ld.w1 = (float)w;
        Ld.off_u = (float)L.offset_u;
        Ld.off_v = (float)L.offset_v;
        Ld.pitch_u = (float)L.pitch_u;
        Ld.pitch_v = (float)L.pitch_v;
        Ld.inv_pitch_u = (float)(1.0 / L.pitch_u);
        Ld.inv_pitch_v = (float)(1.0 / L.pitch_v);
        Ld.glo_u = (float)(0.5 * L.gap_u);
        Ld.ghi_u = (float)(L.pitch_u - 0.5 * L.gap_u);
        Ld.glo_v = (float)(0.5 * L.gap_v);
        Ld.ghi_v = (float)(L.pitch_v - 0.5 * L.gap_v);
        Ld.n_u = L.n_u;
        Ld.n_v = L.n_v;
        Ld.loff = loff;
        Ld.crystal_mat = L.crystal_mat;
        Ld.interval_mat = L.interval_mat;
        loff += L.n_u * L.n_v;
    }
    g.crystals_per_module = loff;
    n_crystals = (int64_t)loff * d->modules_u * d->modules_v * d->n_panels;
    if (n_crystals >= (int64_t)1 << 31) return gpet_fail(GPET_ERR_GEOMETRY, "more than 2^31 crystals");
    g.n_crystals = (int32_t)n_crystals;
    g.R = (float)d->inner_radius_mm;
    g.W = (float)w;
    g.half_u = (float)(0.5 * U);
    g.half_v = (float)(0.5 * V);
    g.msu = (float)d->module_size_u;
    g.msv = (float)d->module_size_v;
    g.mpu = (float)(d->module_size_u + d->module_gap_u);
    g.mpv = (float)(d->module_size_v + d->module_gap_v);
    g.inv_mpu = (float)(1.0 / (d->module_size_u + d->module_gap_u));
    g.inv_mpv = (float)(1.0 / (d->module_size_v + d->module_gap_v));
    for (int m = 0; m < d->n_materials; ++m) {
        const gpet_material &M = d->materials[m];
        g.mu_c511[m] = (float)mu_c511(M);
        g.mu_pe511[m] = (float)(M.mu_total_511_cm * M.photo_frac_511);
    }
    // ring culling parameters (see flight() in device.cuh)
    const double rout = std::sqrt((d->inner_radius_mm + w) * (d->inner_radius_mm + w) + 0.25 * U * U);
    g.R2 = (float)(d->inner_radius_mm * d->inner_radius_mm);
    g.rout2 = (float)(rout * rout * (1.0 + 1e-6));
    g.beta = (float)std::atan2(0.5 * U, d->inner_radius_mm);
    // the culling works with the first panel's angle reduced to [0, 2 pi)
    double phi0 = std::fmod(d->first_angle_rad, 2.0 * M_PI);
    if (phi0 < 0.0) phi0 += 2.0 * M_PI;
    g.phi0 = (float)phi0;
    g.dphi = (float)(2.0 * M_PI / d->n_panels);
    g.inv_dphi = (float)(d->n_panels / (2.0 * M_PI));
    if (posed) {
        std::vector<float> tab;
        const int st = build_poses(d, w, U, V, tab);
        if (st != GPET_OK) return st;
        g.posed = 1;
        g.pose = nullptr;  // device copy placed by the run that uses it
        if (pose_dev) *pose_dev = std::move(tab);
        return GPET_OK;
    }
    std::vector<double> ang(d->n_panels);
    for (int k = 0; k < d->n_panels; ++k) {
        ang[k] = d->first_angle_rad + 2.0 * M_PI * k / d->n_panels;
        g.pc[k] = (float)std::cos(ang[k]);
        g.ps[k] = (float)std::sin(ang[k]);
    }
    for (int a = 0; a < d->n_panels; ++a)
        for (int b = a + 1; b < d->n_panels; ++b)
            if (panels_overlap(d->inner_radius_mm, w, 0.5 * U, ang[a], ang[b]))
                return gpet_fail(GPET_ERR_GEOMETRY, "panels %d and %d overlap (panel width %.3f mm at radius %.3f mm)",
                                 a, b, U, d->inner_radius_mm);
    return GPET_OK;
}

std::string gpet_geometry_key(const gpet_scanner *sc) {
    std::string key(reinterpret_cast<const char *>(&sc->g), sizeof(GeomDev));
    key.append(reinterpret_cast<const char *>(sc->pose_dev.data()), sizeof(float) * sc->pose_dev.size());
    return key;
}

extern "C" int gpet_create_scanner(const gpet_scanner_desc *desc, gpet_scanner **out) {
    if (!out) return gpet_fail(GPET_ERR_INVALID_ARG, "out is NULL");
    GeomDev g;
    int64_t nc = 0;
    std::vector<float> pose_dev;
    int st = gpet_build_geometry(desc, g, nc, &pose_dev);
    if (st != GPET_OK) return st;
    gpet_scanner *sc = new (std::nothrow) gpet_scanner();
    if (!sc) return gpet_fail(GPET_ERR_OOM, "host allocation of the scanner failed");
    sc->desc = *desc;
    sc->layers.assign(desc->layers, desc->layers + desc->n_layers);
    sc->materials.assign(desc->materials, desc->materials + desc->n_materials);
    sc->desc.layers = sc->layers.data();
    sc->desc.materials = sc->materials.data();
    if (desc->panel_poses) {
        sc->poses.assign(desc->panel_poses, desc->panel_poses + 12 * (size_t)desc->n_panels);
        sc->desc.panel_poses = sc->poses.data();
        sc->pose_dev = std::move(pose_dev);
    }
    sc->g = g;
    sc->n_crystals = nc;
    *out = sc;
    return GPET_OK;
}

void free_phantom(gpet_scanner *sc) {
    if (sc->ph_mat) cudaFree(sc->ph_mat);
    if (sc->ph_cdf) cudaFree(sc->ph_cdf);
    if (sc->ph_guide) cudaFree(sc->ph_guide);
    sc->ph_mat = nullptr;
    sc->ph_cdf = nullptr;
    sc->ph_guide = nullptr;
    sc->has_phantom = false;
}

extern "C" void gpet_destroy_scanner(gpet_scanner *sc) {
    if (!sc) return;
    free_phantom(sc);
    delete sc;
}

extern "C" int gpet_scanner_crystals(const gpet_scanner *sc, int64_t *n) {
    if (!sc || !n) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    *n = sc->n_crystals;
    return GPET_OK;
}

extern "C" int gpet_load_phantom(gpet_scanner *sc, int32_t nx, int32_t ny, int32_t nz, const double voxel_mm[3],
                                 const double origin_mm[3], const uint8_t *material_ids, const float *activity,
                                 int32_t n_materials, const gpet_material *materials) {
    if (!sc || !voxel_mm || !origin_mm || !material_ids || !materials)
        return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1) return gpet_fail(GPET_ERR_INVALID_ARG, "grid %d x %d x %d", nx, ny, nz);
    if (n_materials < 1 || n_materials > kMaxMaterials)
        return gpet_fail(GPET_ERR_INVALID_ARG, "phantom n_materials=%d outside [1, %d]", n_materials, kMaxMaterials);
    for (int a = 0; a < 3; ++a)
        if (!(voxel_mm[a] > 0.0) || !std::isfinite(origin_mm[a]))
            return gpet_fail(GPET_ERR_INVALID_ARG, "voxel size must be > 0");
    for (int m = 0; m < n_materials; ++m)
        if (!material_ok(materials[m])) return gpet_fail(GPET_ERR_INVALID_ARG, "phantom material %d out of range", m);
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = 0; i < n; ++i)
        if (material_ids[i] >= n_materials)
            return gpet_fail(GPET_ERR_INVALID_ARG, "voxel %lld has material %d >= %d", (long long)i, material_ids[i],
                             n_materials);
    // the grid must stay clear of the panels (photons never re-enter it after a panel)
    const double xs[2] = {origin_mm[0], origin_mm[0] + nx * voxel_mm[0]};
    const double ys[2] = {origin_mm[1], origin_mm[1] + ny * voxel_mm[1]};
    if (sc->desc.panel_poses) {
        Obb box;
        const double ext[3] = {nx * voxel_mm[0], ny * voxel_mm[1], nz * voxel_mm[2]};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) box.a[i][j] = i == j ? 1.0 : 0.0;
            box.c[i] = origin_mm[i] + 0.5 * ext[i];
            box.e[i] = 0.5 * ext[i];
        }
        const double Wd = sc->g.W, U = 2.0 * sc->g.half_u, V = 2.0 * sc->g.half_v;
        for (int k = 0; k < sc->desc.n_panels; ++k)
            if (boxes_overlap(box, posed_box(sc->poses.data() + 12 * k, Wd, U, V)))
                return gpet_fail(GPET_ERR_GEOMETRY, "phantom grid overlaps posed panel %d", k);
    } else {
        double rmax = 0.0;
        for (double x : xs)
            for (double y : ys) rmax = std::max(rmax, std::sqrt(x * x + y * y));
        if (rmax > sc->desc.inner_radius_mm)
            return gpet_fail(GPET_ERR_GEOMETRY, "phantom reaches radius %.3f mm > ring radius %.3f mm", rmax,
                             sc->desc.inner_radius_mm);
    }
    std::vector<double> cdf;
    double total = 0.0;
    int64_t last = -1;
    if (activity) {
        cdf.resize((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            double a = (double)activity[i];
            if (!std::isfinite(a) || a < 0.0)
                return gpet_fail(GPET_ERR_INVALID_ARG, "voxel %lld activity must be finite and >= 0", (long long)i);
            total += a;
            cdf[(size_t)i] = total;
            if (a > 0.0) last = i;
        }
    }
    free_phantom(sc);
    cudaError_t e = cudaMalloc(&sc->ph_mat, (size_t)n);
    if (e != cudaSuccess) return gpet_cuda_fail(e, "cudaMalloc(phantom)");
    e = cudaMemcpy(sc->ph_mat, material_ids, (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_phantom(sc); return gpet_cuda_fail(e, "cudaMemcpy(phantom)"); }
    if (activity) {
        e = cudaMalloc(&sc->ph_cdf, sizeof(double) * (size_t)n);
        if (e != cudaSuccess) { free_phantom(sc); return gpet_cuda_fail(e, "cudaMalloc(activity)"); }
        e = cudaMemcpy(sc->ph_cdf, cdf.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { free_phantom(sc); return gpet_cuda_fail(e, "cudaMemcpy(activity)"); }
        // guide table: guide[k] = first voxel whose prefix sum lies in bucket >= k
        // (int32 entries: a grid of 2^31 voxels or more is searched without it)
        if (total > 0.0 && n <= (int64_t)INT32_MAX) {
            const int32_t G = (int32_t)std::min<int64_t>(65536, std::max<int64_t>(1, n));
            const double gscale = (double)G / total;
            std::vector<int32_t> guide((size_t)G, (int32_t)(n - 1));
            int32_t k = 0;
            for (int64_t i = 0; i < n && k < G; ++i) {
                const int64_t b = std::min<int64_t>((int64_t)(cdf[(size_t)i] * gscale), G - 1);
                while (k <= b && k < G) guide[(size_t)k++] = (int32_t)i;
            }
            e = cudaMalloc(&sc->ph_guide, sizeof(int32_t) * (size_t)G);
            if (e != cudaSuccess) { free_phantom(sc); return gpet_cuda_fail(e, "cudaMalloc(guide)"); }
            e = cudaMemcpy(sc->ph_guide, guide.data(), sizeof(int32_t) * (size_t)G, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { free_phantom(sc); return gpet_cuda_fail(e, "cudaMemcpy(guide)"); }
            sc->ph_buckets = G;
            sc->ph_gscale = gscale;
        }
    }
    sc->has_phantom = true;
    sc->ph_n[0] = nx; sc->ph_n[1] = ny; sc->ph_n[2] = nz;
    for (int a = 0; a < 3; ++a) { sc->ph_voxel[a] = voxel_mm[a]; sc->ph_origin[a] = origin_mm[a]; }
    sc->ph_materials.assign(materials, materials + n_materials);
    sc->ph_total = total;
    sc->ph_last_active = last;
    return GPET_OK;
}

// ---------------------------------------------------------------------------
// job description for the kernels
// ---------------------------------------------------------------------------
int gpet_make_job(const gpet_scanner *sc, const gpet_source *src, const gpet_digitizer *dg, uint64_t n_decays,
                  uint64_t seed, JobDev &J, uint64_t h_begin, uint64_t h_end) {
    if (!sc || !src || !dg) return gpet_fail(GPET_ERR_INVALID_ARG, "NULL argument");
    if (n_decays == 0) return gpet_fail(GPET_ERR_INVALID_ARG, "n_decays must be > 0");
    if (h_end == 0) h_end = n_decays;
    if (h_end > n_decays || h_begin >= h_end)
        return gpet_fail(GPET_ERR_INVALID_ARG, "history range [%llu, %llu) outside the %llu-decay run",
                         (unsigned long long)h_begin, (unsigned long long)h_end, (unsigned long long)n_decays);
    if (!(src->activity_bq > 0.0) || !std::isfinite(src->activity_bq))
        return gpet_fail(GPET_ERR_INVALID_ARG, "activity must be > 0");
    if (src->kind < 0 || src->kind > 2) return gpet_fail(GPET_ERR_INVALID_ARG, "source kind %d", src->kind);
    if (src->kind == GPET_SOURCE_PHANTOM && (!sc->has_phantom || !sc->ph_cdf || !(sc->ph_total > 0.0)))
        return gpet_fail(GPET_ERR_INVALID_ARG, "phantom source without a loaded activity map");
    if (!(dg->e_cut_kev >= kXsEmin) || !(dg->e_cut_kev < 511.0))
        return gpet_fail(GPET_ERR_INVALID_ARG, "e_cut_kev must lie in [%g, 511)", (double)kXsEmin);
    if (!(dg->fwhm_at_511 >= 0.0) || !(dg->coinc_window_ns >= 0.0) || !(dg->e_hi_kev >= dg->e_lo_kev) ||
        !(dg->doi_fwhm_mm >= 0.0))
        return gpet_fail(GPET_ERR_INVALID_ARG, "digitizer settings out of range");
    const double span = (double)n_decays / src->activity_bq * 1e12;
    // time stamps are uint64 ps; a launch of several jobs checks that its
    // longest acquisition also fits beside the job bits of the sort key
    if (!(span < 0x1p62)) return gpet_fail(GPET_ERR_INVALID_ARG, "acquisition longer than 2^62 ps (53 days)");
    if (src->kind == GPET_SOURCE_PENCIL) {
        const double nn = src->dir[0] * src->dir[0] + src->dir[1] * src->dir[1] + src->dir[2] * src->dir[2];
        if (!(std::fabs(nn - 1.0) < 1e-6)) return gpet_fail(GPET_ERR_INVALID_ARG, "pencil direction must be a unit vector");
    }
    std::memset(&J, 0, sizeof(J));
    J.geom = 0;
    J.seed = seed;
    J.n_decays = n_decays;
    J.h_base = h_begin;
    J.n_hist = h_end - h_begin;
    J.t_span_ps = (uint64_t)std::llround(span);
    J.src_kind = src->kind;
    for (int a = 0; a < 3; ++a) {
        J.src_pos[a] = (float)src->pos_mm[a];
        J.src_dir[a] = (float)src->dir[a];
    }
    J.e_cut = (float)dg->e_cut_kev;
    J.e_lo = (float)dg->e_lo_kev;
    J.e_hi = (float)dg->e_hi_kev;
    J.sig_k = (float)(dg->fwhm_at_511 / (2.0 * std::sqrt(2.0 * std::log(2.0))));
    J.sig_doi = (float)(dg->doi_fwhm_mm / (2.0 * std::sqrt(2.0 * std::log(2.0))));
    if (sc->has_phantom) {
        J.has_phantom = 1;
        J.ph_nx = sc->ph_n[0]; J.ph_ny = sc->ph_n[1]; J.ph_nz = sc->ph_n[2];
        J.ph_nmat = (int32_t)sc->ph_materials.size();
        for (int a = 0; a < 3; ++a) {
            J.ph_origin[a] = (float)sc->ph_origin[a];
            J.ph_voxel[a] = (float)sc->ph_voxel[a];
            J.ph_inv_voxel[a] = (float)(1.0 / sc->ph_voxel[a]);
            J.ph_hi[a] = (float)(sc->ph_origin[a] + sc->ph_n[a] * sc->ph_voxel[a]);
        }
        for (size_t m = 0; m < sc->ph_materials.size(); ++m) {
            J.ph_mu_c511[m] = (float)mu_c511(sc->ph_materials[m]);
            J.ph_mu_pe511[m] = (float)(sc->ph_materials[m].mu_total_511_cm * sc->ph_materials[m].photo_frac_511);
        }
        J.ph_mat = sc->ph_mat;
        J.ph_cdf = sc->ph_cdf;
        J.ph_guide = sc->ph_guide;
        J.ph_buckets = sc->ph_buckets;
        J.ph_gscale = sc->ph_gscale;
        J.ph_total = sc->ph_total;
        J.ph_n = (int64_t)sc->ph_n[0] * sc->ph_n[1] * sc->ph_n[2];
        J.ph_last_active = sc->ph_last_active;
    }
    return GPET_OK;
}
