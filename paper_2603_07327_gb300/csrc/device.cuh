// device.cuh -- device-side building blocks of the multi-layer photon-pair
// transport: geometry descriptor, Philox4x32-10 streams, cross sections,
// Klein-Nishina sampling, hierarchy location and panel flight.
//
// Paper anchors (arxiv 2603.07327): Sec. 2.1 / Fig. 1 for the four-level
// panel -> module -> layer -> crystal description, the repetition mode, the
// line-plane flight from the phantom to a panel, the panel-local frame, the
// Woodcock free-path sampling and the layer-selection step; Sec. 2.3 for the
// source (back-to-back pairs, no positron range) and the digitizer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gpet {

// One single as the transport kernels append it: a 48-byte record, so that the
// time-order gather reads each single from two 32-byte sectors.
struct __align__(16) RawSingle {
    uint64_t t, h;        // time (ps), history
    int32_t unit, panel, job;
    float e, e_raw, doi;  // blurred and raw energy (keV), blurred depth (mm)
    uint32_t pad[2];
};
static_assert(sizeof(RawSingle) == 48, "RawSingle layout");

constexpr uint32_t kFullMask = 0xFFFFFFFFu;
constexpr int kMaxPanels = 64;
constexpr int kMaxLayers = 8;
constexpr int kMaxMaterials = 8;
constexpr int kXsIntervals = 4096;       // log-E intervals of the Compton ratio table
constexpr float kXsEmin = 1.0f;          // keV, lower end of the table
constexpr int kMaxSteps = 1000;          // per photon and region; cap -> GPET_ERR_TIMEOUT
constexpr int kMaxTrials = 1000;         // Kahn rejection cap
constexpr float kE0 = 511.0f;            // annihilation photon energy (keV)
constexpr float kInvMec2 = 1.0f / 510.99895f;
constexpr float kInvCmmPerPs = 1.0f / 0.299792458f;  // ps per mm
constexpr float kEfxScale = 1048576.0f;  // tally energy unit 2^-20 keV

enum : uint32_t { kTagSource = 1u, kTagPhantom = 2u, kTagDetector = 3u, kTagDigi = 4u };

// device status codes (host maps them to GPET_ERR_*)
// kStatusBadPhase: a history in a phase no event handles (an internal error);
// the history is dropped, so no event loop can spin on it.
// kStatusSortStall: a radix-sort tile copy or look-back did not complete
// within the wait limit, or a pass computed an offset past its keys; the sort
// stops (or skips the write) and its output is invalid (an internal error).
// kStatusLiveStall: a live launch found no new work and no end of the work
// queue for the whole idle-wait limit; its CTAs stop (an internal error).
enum : int { kStatusOk = 0, kStatusTimeout = 1, kStatusOverflow = 2, kStatusBadPhase = 4, kStatusSortStall = 8,
             kStatusLiveStall = 16 };

// ---------------------------------------------------------------------------
// geometry descriptor (FP32, one per scanner design)
// ---------------------------------------------------------------------------
struct LayerDev {
    float w0, w1;                   // crystal depth range [w0, w1) in the panel frame
    float off_u, off_v;             // crystal grid offset inside the module
    float pitch_u, pitch_v;
    float inv_pitch_u, inv_pitch_v;
    float glo_u, ghi_u, glo_v, ghi_v;  // crystal occupies [glo, ghi) of its cell
    int32_t n_u, n_v, loff;         // crystals per row / column, id offset in the module
    int32_t crystal_mat, interval_mat;  // interval_mat also fills the radial gap in front
};

// Descriptors start on 128-byte lines: a live launch appends descriptors while
// its kernel runs, and no line may hold a published and an unpublished one
// (the L1 cache could otherwise keep the unpublished bytes of a line it loaded).
struct __align__(128) GeomDev {
    int32_t n_panels, n_layers, n_materials, modules_u, modules_v, readout_level;
    int32_t crystals_per_module, n_crystals;
    float R, W, half_u, half_v;     // inner radius, panel depth, half extents
    float msu, msv, mpu, mpv, inv_mpu, inv_mpv;  // module size, module pitch (size + gap)
    float mu_c511[kMaxMaterials];   // Compton coefficient at 511 keV (1/cm)
    float mu_pe511[kMaxMaterials];  // photoelectric coefficient at 511 keV (1/cm)
    float pc[kMaxPanels], ps[kMaxPanels];  // cos / sin of each panel's angle
    // ring culling: every panel box lies in the annulus R^2 <= r^2 <= rout2 and
    // inside its angular sector |phi - phi_k| <= beta (phi_k = phi0 + k dphi)
    float R2, rout2, beta, phi0, dphi, inv_dphi;
    // non-repetition mode (posed = 1): per panel 4 float4 in global memory --
    // (w axis, w.o), (u axis, u.o), (v axis, v.o), (o, 0) with o the centre of
    // the inner face; the ring fields above are then unused
    const float4 *pose;
    int32_t posed, pose_pad;
    LayerDev layers[kMaxLayers];
};
static_assert(sizeof(GeomDev) % 16 == 0, "GeomDev is copied in words and staged in shared memory");

// one simulation job: a scanner design (index into the geometry table), a
// source and its digitizer settings
struct __align__(128) JobDev {
    uint64_t seed, n_decays, t_span_ps;
    uint64_t h_base, n_hist;          // histories [h_base, h_base + n_hist) of the run
    int32_t geom, src_kind;
    float src_pos[3], src_dir[3];
    float e_cut, e_lo, e_hi, sig_k;   // sig_k = fwhm_511 / (2 sqrt(2 ln 2))
    float sig_doi, pad_doi;           // depth blur sigma (mm)
    // phantom (has_phantom = 0 when none)
    int32_t has_phantom, ph_nx, ph_ny, ph_nz, ph_nmat;
    float ph_origin[3], ph_voxel[3], ph_inv_voxel[3], ph_hi[3];
    float ph_mu_c511[kMaxMaterials], ph_mu_pe511[kMaxMaterials];
    const uint8_t *ph_mat;
    const double *ph_cdf;             // activity prefix sums in voxel order
    const int32_t *ph_guide;          // guide table: first voxel of each bucket of the total
    double ph_total, ph_gscale;       // gscale = buckets / total
    int64_t ph_n, ph_last_active;
    int32_t ph_buckets, ph_pad;
    // per-crystal tallies of this job
    unsigned long long *tally_count, *tally_efx;
    // singles of this job: NULL s_raw appends them to the launch's buffer;
    // else to the job's own (a served request split over several launches
    // gathers its singles there), counted in *n_singles up to s_cap and
    // recorded as job 0 (the one job of the run that owns that buffer)
    RawSingle *s_raw;
    unsigned long long *n_singles;
    unsigned long long s_cap;
    uint64_t *s_keys;                 // the sort keys of that buffer (its time stamps)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += W0; k.y += W1; }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// draw block (history, tag, photon, step, sub) under key = seed
__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t h, uint32_t tag, uint32_t gamma, uint32_t step,
                                      uint32_t sub) {
    return philox4x32_10(make_uint4((uint32_t)h, (uint32_t)(h >> 32),
                                    (tag << 28) | ((gamma & 1u) << 27) | (step & 0x07FFFFFFu), sub),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// uniform (k + 1/2) 2^-23 in (0,1) from the top 23 bits (exact in FP32)
__device__ __forceinline__ float u01(uint32_t w) {
    return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// ---------------------------------------------------------------------------
// cross sections: mu_C(E) = mu_C(511) * g(E), g = sigma_KN(E)/sigma_KN(511) from a
// log-E table; mu_pe(E) = mu_pe(511) * (511/E)^3
// ---------------------------------------------------------------------------
struct Xs {
    float g;    // Compton ratio
    float r3;   // (511/E)^3
};

__device__ __forceinline__ Xs xs_at(float E, const float *__restrict__ gtab, float ln_emin, float inv_h) {
    Xs x;
    if (E >= kE0) {
        x.g = 1.0f;
        x.r3 = 1.0f;
        return x;
    }
    float t = (__logf(E) - ln_emin) * inv_h;
    t = fmaxf(t, 0.0f);
    int i = min((int)t, kXsIntervals - 1);
    float f = t - (float)i;
    float g0 = __ldg(gtab + i), g1 = __ldg(gtab + i + 1);
    x.g = fmaf(f, g1 - g0, g0);
    float r = kE0 / E;
    x.r3 = r * r * r;
    return x;
}

__device__ __forceinline__ float mu_total(float c511, float pe511, const Xs &x) {
    return fmaf(c511, x.g, pe511 * x.r3);
}

// ---------------------------------------------------------------------------
// Kahn's rejection sampling of Klein-Nishina
// ---------------------------------------------------------------------------
// one trial from one Philox block: candidate xm1 = E/E' - 1 and its acceptance
__device__ __forceinline__ bool kahn_try(const uint4 r, float k, float a, float b, float &xm1) {
    const float r1 = u01(r.x), r2 = u01(r.y), r3 = u01(r.z);
    bool accept;
    if (r1 * b <= a) {
        xm1 = 2.0f * k * r2;
        const float eta = 1.0f + xm1;
        accept = r3 * eta * eta <= 4.0f * xm1;
    } else {
        const float den = fmaf(2.0f * k, r2, 1.0f);
        xm1 = 2.0f * k * (1.0f - r2) / den;
        const float eta = 1.0f + xm1;
        const float c = 1.0f - xm1 / k;
        accept = 2.0f * r3 <= fmaf(c, c, 1.0f / eta);
    }
    return accept;
}

// Kahn's rejection sampling of Klein-Nishina; returns trials (> 0) or -1.
// Trials are evaluated two at a time (independent Philox blocks, so the two
// chains overlap); the first accepted one in trial order is returned.
__device__ __forceinline__ int kahn_sample(uint64_t seed, uint64_t h, uint32_t tag, uint32_t gamma, uint32_t step,
                                           float E, float &xm1_out) {
    const float k = E * kInvMec2;
    const float a = 1.0f + 2.0f * k;
    const float b = 9.0f + 2.0f * k;
    for (int trial = 0; trial < kMaxTrials; trial += 2) {
        const uint4 ra = draw(seed, h, tag, gamma, step, 1u + (uint32_t)trial);
        const uint4 rb = draw(seed, h, tag, gamma, step, 2u + (uint32_t)trial);
        float xa, xb;
        const bool acc_a = kahn_try(ra, k, a, b, xa);
        const bool acc_b = kahn_try(rb, k, a, b, xb);
        if (acc_a) { xm1_out = xa; return trial + 1; }
        if (acc_b) { xm1_out = xb; return trial + 2; }
    }
    return -1;
}

// rotate (a, b, c) [third component = scanner axis] by polar (cos ct, 1-cos omc) and
// azimuth 2 pi u; frame-equivariant under rotations about the axis
__device__ __forceinline__ void rotate_dir(float &a, float &b, float &c, float omc, float u_phi) {
    const float ct = 1.0f - omc;
    const float st = sqrtf(fmaxf(omc * (2.0f - omc), 0.0f));
    float sp, cp;
    sincospif(2.0f * u_phi, &sp, &cp);
    if (fabsf(c) < 0.99999f) {
        // transverse norm from the transverse components (= sqrt(1 - c^2) for a
        // unit vector, without the cancellation of 1 - c^2 near the axis)
        const float q = sqrtf(fmaf(a, a, b * b));
        const float iq = 1.0f / q;
        const float na = a * ct + st * (a * c * cp - b * sp) * iq;
        const float nb = b * ct + st * (b * c * cp + a * sp) * iq;
        const float nc = c * ct - st * q * cp;
        a = na; b = nb; c = nc;
    } else {
        const float sg = c > 0.0f ? 1.0f : -1.0f;
        a = st * cp;
        b = st * sp;
        c = sg * ct;
    }
}

// ---------------------------------------------------------------------------
// hierarchy location in the panel frame (layer selection, module, crystal)
// ---------------------------------------------------------------------------
struct Loc {
    int32_t layer, module, crystal;   // crystal = global id or -1
    int32_t mat;
};

__device__ __forceinline__ Loc locate(const GeomDev &g, int k, float w, float u, float v) {
    Loc L;
    L.layer = -1; L.module = -1; L.crystal = -1;
    // layer-selection step: the layer whose depth range holds w
    int l = -1, owner = g.n_layers - 1;
    for (int j = 0; j < g.n_layers; ++j) {
        if (w < g.layers[j].w0) { owner = j; break; }
        if (w < g.layers[j].w1) { l = j; break; }
    }
    if (l < 0) {
        L.mat = g.layers[owner].interval_mat;
        return L;
    }
    const LayerDev &Ly = g.layers[l];
    L.layer = l;
    L.mat = Ly.interval_mat;
    const float au = u + g.half_u, av = v + g.half_v;
    const int mu = (int)floorf(au * g.inv_mpu), mv = (int)floorf(av * g.inv_mpv);
    if (mu < 0 || mu >= g.modules_u || mv < 0 || mv >= g.modules_v) return L;
    const float a_u = fmaf(-(float)mu, g.mpu, au), a_v = fmaf(-(float)mv, g.mpv, av);
    if (a_u >= g.msu || a_v >= g.msv) return L;
    L.module = mv * g.modules_u + mu;
    const float bu = a_u - Ly.off_u, bv = a_v - Ly.off_v;
    const int iu = (int)floorf(bu * Ly.inv_pitch_u), iv = (int)floorf(bv * Ly.inv_pitch_v);
    if (iu < 0 || iu >= Ly.n_u || iv < 0 || iv >= Ly.n_v) return L;
    const float cu = fmaf(-(float)iu, Ly.pitch_u, bu), cv = fmaf(-(float)iv, Ly.pitch_v, bv);
    if (cu < Ly.glo_u || cu >= Ly.ghi_u || cv < Ly.glo_v || cv >= Ly.ghi_v) return L;
    L.mat = Ly.crystal_mat;
    L.crystal = ((k * g.modules_v + mv) * g.modules_u + mu) * g.crystals_per_module + Ly.loff + iv * Ly.n_u + iu;
    return L;
}

// distance along (dw, du, dv) from an inside point to the panel box exit
__device__ __forceinline__ float panel_exit(const GeomDev &g, float w, float u, float v, float dw, float du, float dv) {
    float t = 3.0e38f;
    if (dw > 0.0f) t = fminf(t, (g.W - w) / dw); else if (dw < 0.0f) t = fminf(t, -w / dw);
    if (du > 0.0f) t = fminf(t, (g.half_u - u) / du); else if (du < 0.0f) t = fminf(t, (-g.half_u - u) / du);
    if (dv > 0.0f) t = fminf(t, (g.half_v - v) / dv); else if (dv < 0.0f) t = fminf(t, (-g.half_v - v) / dv);
    return fmaxf(t, 0.0f);
}

// slab test of the ray against panel k's box in its own frame; keeps the
// nearest entry (ties to the lower panel index)
__device__ __forceinline__ void panel_slab(const GeomDev &g, int k, float x, float y, float z, float dx, float dy,
                                           float dz, int &best, float &bi, float &bo) {
    {
        const float c = g.pc[k], s = g.ps[k];
        const float w0 = fmaf(x, c, y * s) - g.R;
        const float dw = fmaf(dx, c, dy * s);
        // behind the inner face and moving away: no entry
        if (w0 < 0.0f && dw <= 0.0f) return;
        const float u0 = fmaf(-x, s, y * c);
        const float du = fmaf(-dx, s, dy * c);
        float tmin = -3.0e38f, tmax = 3.0e38f;
        bool miss = false;
        // w slab [0, W]
        if (dw != 0.0f) {
            const float i = 1.0f / dw;
            const float t1 = -w0 * i, t2 = (g.W - w0) * i;
            tmin = fmaxf(tmin, fminf(t1, t2));
            tmax = fminf(tmax, fmaxf(t1, t2));
        } else if (w0 < 0.0f || w0 > g.W) miss = true;
        if (du != 0.0f) {
            const float i = 1.0f / du;
            const float t1 = (-g.half_u - u0) * i, t2 = (g.half_u - u0) * i;
            tmin = fmaxf(tmin, fminf(t1, t2));
            tmax = fminf(tmax, fmaxf(t1, t2));
        } else if (u0 < -g.half_u || u0 > g.half_u) miss = true;
        if (dz != 0.0f) {
            const float i = 1.0f / dz;
            const float t1 = (-g.half_v - z) * i, t2 = (g.half_v - z) * i;
            tmin = fmaxf(tmin, fminf(t1, t2));
            tmax = fminf(tmax, fmaxf(t1, t2));
        } else if (z < -g.half_v || z > g.half_v) miss = true;
        tmin = fmaxf(tmin, 0.0f);
        if (!miss && tmin < tmax && (tmin < bi || (tmin == bi && k < best))) {
            best = k;
            bi = tmin;
            bo = tmax;
        }
    }
}

// slab test of the ray against posed panel k (non-repetition mode): the
// same box test in the panel's own (w, u, v) frame, read from its pose
__device__ __forceinline__ void panel_slab_posed(const GeomDev &g, int k, float x, float y, float z, float dx,
                                                 float dy, float dz, int &best, float &bi, float &bo) {
    const float4 aw = __ldg(g.pose + 4 * k), au = __ldg(g.pose + 4 * k + 1), av = __ldg(g.pose + 4 * k + 2);
    const float w0 = fmaf(x, aw.x, fmaf(y, aw.y, fmaf(z, aw.z, -aw.w)));
    const float dw = fmaf(dx, aw.x, fmaf(dy, aw.y, dz * aw.z));
    if (w0 < 0.0f && dw <= 0.0f) return;  // behind the inner face and moving away
    const float u0 = fmaf(x, au.x, fmaf(y, au.y, fmaf(z, au.z, -au.w)));
    const float du = fmaf(dx, au.x, fmaf(dy, au.y, dz * au.z));
    const float v0 = fmaf(x, av.x, fmaf(y, av.y, fmaf(z, av.z, -av.w)));
    const float dv = fmaf(dx, av.x, fmaf(dy, av.y, dz * av.z));
    float tmin = -3.0e38f, tmax = 3.0e38f;
    bool miss = false;
    if (dw != 0.0f) {
        const float i = 1.0f / dw;
        const float t1 = -w0 * i, t2 = (g.W - w0) * i;
        tmin = fmaxf(tmin, fminf(t1, t2));
        tmax = fminf(tmax, fmaxf(t1, t2));
    } else if (w0 < 0.0f || w0 > g.W) miss = true;
    if (du != 0.0f) {
        const float i = 1.0f / du;
        const float t1 = (-g.half_u - u0) * i, t2 = (g.half_u - u0) * i;
        tmin = fmaxf(tmin, fminf(t1, t2));
        tmax = fminf(tmax, fmaxf(t1, t2));
    } else if (u0 < -g.half_u || u0 > g.half_u) miss = true;
    if (dv != 0.0f) {
        const float i = 1.0f / dv;
        const float t1 = (-g.half_v - v0) * i, t2 = (g.half_v - v0) * i;
        tmin = fmaxf(tmin, fminf(t1, t2));
        tmax = fminf(tmax, fmaxf(t1, t2));
    } else if (v0 < -g.half_v || v0 > g.half_v) miss = true;
    tmin = fmaxf(tmin, 0.0f);
    if (!miss && tmin < tmax && (tmin < bi || (tmin == bi && k < best))) {
        best = k;
        bi = tmin;
        bo = tmax;
    }
}

// atan2 from the odd polynomial of Abramowitz & Stegun 4.4.47 (|error| <= 1e-5
// rad on [-1, 1]) with octant reduction; used only to pick candidate panels,
// where a 1e-3 rad margin absorbs its error
__device__ __forceinline__ float atan2_as(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float t2 = t * t;
    float r = fmaf(t2, 0.0208351f, -0.0851330f);
    r = fmaf(t2, r, 0.1801410f);
    r = fmaf(t2, r, -0.3302995f);
    r = fmaf(t2, r, 0.9998660f);
    r *= t;
    if (ay > ax) r = 1.57079633f - r;
    if (x < 0.0f) r = 3.14159265f - r;
    return y < 0.0f ? -r : r;
}

constexpr int kFlightScreened = -2;  // flight() result: no panel, decided without slab tests

// Slab-test the panels whose angular sector can meet the azimuths the ray
// sweeps between t = ta and t = tb (a stretch inside the annulus that holds
// all panel boxes; along a line the azimuth is monotonic and the sweep is
// shorter than pi).  Panel k can be entered there only if its centre angle
// k*dphi lies within beta of the swept interval; 1e-3 rad of margin covers
// FP32 rounding.
__device__ __forceinline__ void flight_sector(const GeomDev &g, float x, float y, float z, float dx, float dy,
                                              float dz, float ta, float tb, int skip, int &best, float &bi,
                                              float &bo) {
    const float p1 = atan2_as(fmaf(ta, dy, y), fmaf(ta, dx, x)) - g.phi0;
    float p2 = atan2_as(fmaf(tb, dy, y), fmaf(tb, dx, x)) - g.phi0;
    // unwrap p2 next to p1
    if (p2 - p1 > 3.14159265f) p2 -= 6.28318531f;
    else if (p1 - p2 > 3.14159265f) p2 += 6.28318531f;
    const float lo = fminf(p1, p2) - g.beta - 1e-3f, hi = fmaxf(p1, p2) + g.beta + 1e-3f;
    const int jlo = (int)ceilf(lo * g.inv_dphi), jhi = (int)floorf(hi * g.inv_dphi);
    // jlo mod n by a float floor: (jlo + 1/2) / n lies at least 1/(2n) from an
    // integer, far beyond the rounding of the quotient for the |jlo| < 4n that
    // phi0 in [0, 2 pi) allows; then step through the panels with a wrap
    const int n = g.n_panels;
    int k = jlo - n * (int)floorf(((float)jlo + 0.5f) * __frcp_rn((float)n));
    for (int j = jlo; j <= jhi && j < jlo + n; ++j) {
        if (k != skip) panel_slab(g, k, x, y, z, dx, dy, dz, best, bi, bo);
        k = k + 1 == n ? 0 : k + 1;
    }
}

// Axial screen of a ray that starts inside the ring (c0 = x^2 + y^2 below
// 0.9999 R^2): true when it runs parallel to the axis, or when it is beyond
// the panels' axial extent (1e-3 mm margin) on reaching the circle R and moving
// away; t1 receives the distance to that circle.
__device__ __forceinline__ bool inside_screened(const GeomDev &g, float z, float dz, float a, float b, float c0,
                                                float &t1) {
    if (a <= 0.0f) return true;
    const float d1 = g.R2 - c0;
    const float s1 = sqrtf(fmaf(b, b, a * d1));
    t1 = b > 0.0f ? __fdividef(d1, b + s1) : __fdividef(s1 - b, a);
    const float z1 = fmaf(t1, dz, z);
    return (z1 > g.half_v + 1e-3f && dz >= 0.0f) || (z1 < -g.half_v - 1e-3f && dz <= 0.0f);
}

// The screen flight() applies first to a ray from (x, d): the same test,
// for deciding at a photon's start that its flight cannot reach a panel.
__device__ __forceinline__ bool start_screened(const GeomDev &g, float x, float y, float z, float dx, float dy,
                                               float dz) {
    if (g.posed || g.n_panels <= 2) return false;
    const float c0 = fmaf(x, x, y * y);
    if (!(c0 < g.R2 * 0.9999f)) return false;
    const float a = fmaf(dx, dx, dy * dy), b = fmaf(x, dx, y * dy);
    float t1;
    return inside_screened(g, z, dz, a, b, c0, t1);
}

// Line-plane flight (Sec. 2.1): nearest panel entered along (x, d), skipping
// `skip`.  Every panel box lies in the annulus between the circle of radius
// R (every inner face is tangent to it) and the circle through the outer
// corners, so only the stretches of the ray inside that annulus matter: one
// for a ray that starts inside R, at most two (before and after it passes
// inside R) for one that starts in or beyond the annulus.  Only panels whose
// sector meets the azimuths of those stretches are slab-tested, which gives
// the same result as testing all panels.
__device__ __forceinline__ int flight(const GeomDev &g, float x, float y, float z, float dx, float dy, float dz,
                                      int skip, float &t_in, float &t_out) {
    int best = -1;
    float bi = 3.0e38f, bo = 0.0f;
    const float c0 = fmaf(x, x, y * y);
    const float a = fmaf(dx, dx, dy * dy);
    const float b = fmaf(x, dx, y * dy);
    if (g.posed) {
        // panels placed one by one: no ring symmetry to cull with
        for (int k = 0; k < g.n_panels; ++k) {
            if (k == skip) continue;
            panel_slab_posed(g, k, x, y, z, dx, dy, dz, best, bi, bo);
        }
    } else if (g.n_panels <= 2) {
        for (int k = 0; k < g.n_panels; ++k) {
            if (k == skip) continue;
            panel_slab(g, k, x, y, z, dx, dy, dz, best, bi, bo);
        }
    } else if (c0 < g.R2 * 0.9999f) {
        // parallel to the axis, or axially beyond the panels when it reaches
        // the annulus: screened; else t1 = exit distance of the circle R
        float t1 = 0.0f;
        if (inside_screened(g, z, dz, a, b, c0, t1)) {
            t_in = bi;
            t_out = bo;
            return kFlightScreened;
        }
        // exit distance of the circle R_out (stable root, c0 < R^2)
        const float d2 = g.rout2 - c0;
        const float s2 = sqrtf(fmaf(b, b, a * d2));
        const float t2 = b > 0.0f ? __fdividef(d2, b + s2) : __fdividef(s2 - b, a);
        flight_sector(g, x, y, z, dx, dy, dz, t1, t2, skip, best, bi, bo);
    } else if (a > 0.0f) {
        // start in or beyond the annulus; its circles are widened by 1e-4 in
        // r^2 so that rounding can only add candidates
        const float ro2 = g.rout2 * 1.0001f, ri2 = g.R2 * 0.9999f;
        const float cA = c0 - ro2;
        const float DA = fmaf(b, b, -a * cA);
        if (cA > 0.0f && (b >= 0.0f || DA <= 0.0f)) {
            t_in = bi;
            t_out = bo;
            return kFlightScreened;  // beyond the outer circle and never coming back inside it
        }
        const float sA = sqrtf(fmaxf(DA, 0.0f));
        // roots tA <= tB of the outer circle (stable forms)
        const float tB = b > 0.0f ? __fdividef(-cA, b + sA) : __fdividef(sA - b, a);
        const float tA = b > 0.0f ? __fdividef(-(b + sA), a) : __fdividef(cA, sA - b);
        const float t0 = fmaxf(tA, 0.0f);
        const float cR = c0 - ri2;
        const float DR = fmaf(b, b, -a * cR);
        if (b < 0.0f && DR > 0.0f) {
            // passes inside the inner circle between tC and tD
            const float sR = sqrtf(DR);
            const float tC = __fdividef(cR, sR - b), tD = __fdividef(sR - b, a);
            flight_sector(g, x, y, z, dx, dy, dz, t0, tC, skip, best, bi, bo);
            flight_sector(g, x, y, z, dx, dy, dz, tD, tB, skip, best, bi, bo);
        } else {
            flight_sector(g, x, y, z, dx, dy, dz, t0, tB, skip, best, bi, bo);
        }
    } else {
        for (int k = 0; k < g.n_panels; ++k) {
            if (k == skip) continue;
            panel_slab(g, k, x, y, z, dx, dy, dz, best, bi, bo);
        }
    }
    t_in = bi;
    t_out = bo;
    return best;
}

}  // namespace gpet
