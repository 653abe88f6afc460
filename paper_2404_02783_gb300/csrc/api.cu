// C ABI of the particle-mesh library (include/pm.h): argument checks, workspace
// carving, host FP64 tables and the orchestration of the device passes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "host_cosmo.h"
#include "internal.h"
#include "particles.h"

using namespace pm;

namespace {

thread_local std::string g_err;

pm_status fail(pm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define PM_CK(expr)                                                                             \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return fail(PM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define PM_TRY(expr)                      \
    do {                                  \
        pm_status s_ = (expr);            \
        if (s_ != PM_OK) return s_;       \
    } while (0)

bool pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }
size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

pm_status check_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(PM_ERR_UNSUPPORTED, "no CUDA device");
    }
    int major = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess || major != 10) {
        cudaGetLastError();
        return fail(PM_ERR_UNSUPPORTED, "needs a Blackwell (sm_10x) GPU; this library is built for sm_103a");
    }
    PM_CK(ensure_device_tables());
    return PM_OK;
}

struct Layout {
    size_t x = 0, p = 0, rho = 0, spec[3] = {0, 0, 0}, force[3] = {0, 0, 0};
    size_t phi_old = 0, island = 0, amp = 0, bin_of = 0, wtab = 0, acc = 0, mid = 0, total = 0;
    bool gr = false, has_island = false, has_mid = false;
};

constexpr int kMaxBins = 256;
// Mean of the particle density in mesh-cell mass units (np^3 particles of mass (n / np)^3 on
// n^3 cells), subtracted as the forward transform loads it: the operators drop the zero mode,
// and the transform's FP32 rounding then scales with delta instead of with 1 + delta.
constexpr double kDensityMean = 1.0;

pm_status validate(const pm_config* c) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null config");
    if (!pow2(c->np) || c->np < 16 || c->np > 1024) return fail(PM_ERR_INVALID_ARG, "np must be a power of two in 16..1024");
    if (!pow2(c->nmesh) || c->nmesh < 16 || c->nmesh > 1024)
        return fail(PM_ERR_INVALID_ARG, "nmesh must be a power of two in 16..1024");
    if (c->nmesh % c->np) return fail(PM_ERR_INVALID_ARG, "nmesh must be a multiple of np");
    if (!(c->box > 0)) return fail(PM_ERR_INVALID_ARG, "box must be positive");
    if (!(c->omega_m > 0 && c->omega_m <= 1 && c->h > 0 && c->sigma8 > 0 && c->omega_b >= 0 && c->omega_b < c->omega_m))
        return fail(PM_ERR_INVALID_ARG, "bad cosmological parameters");
    if (!(c->a_init > 0 && c->a_final > c->a_init)) return fail(PM_ERR_INVALID_ARG, "need 0 < a_init < a_final");
    if (c->n_steps < 1) return fail(PM_ERR_INVALID_ARG, "n_steps must be >= 1");
    if (c->mode != PM_NEWTON && c->mode != PM_GR_POISSON) return fail(PM_ERR_INVALID_ARG, "bad mode");
    if (c->precision != PM_FP32_FIXED && c->precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    if (c->n_lo < 0 || 2 * c->n_lo >= c->nmesh) return fail(PM_ERR_INVALID_ARG, "n_lo must be in [0, nmesh/2)");
    if (c->gradient != PM_GRAD_SPECTRAL && c->gradient != PM_GRAD_FD1) return fail(PM_ERR_INVALID_ARG, "bad gradient");
    if (c->stepping != PM_STEP_INTEGRALS && c->stepping != PM_STEP_GROWTH)
        return fail(PM_ERR_INVALID_ARG, "bad stepping");
    return PM_OK;
}

// Leapfrog factors of a run: the kick from a0 to a1 with the force taken at a_force, the
// drift from a0 to a1 with the momenta held at a_mom (the FP64 integrals ignore both).
double kick_factor(const pm_config& cfg, const pmhost::Cosmo& co, double a0, double a1, double a_force) {
    return cfg.stepping == PM_STEP_GROWTH ? pmhost::kick_growth(co, a0, a1, a_force)
                                          : pmhost::kick_integral(co, a0, a1);
}
double drift_factor(const pm_config& cfg, const pmhost::Cosmo& co, double a0, double a1, double a_mom) {
    return cfg.stepping == PM_STEP_GROWTH ? pmhost::drift_growth(co, a0, a1, a_mom)
                                          : pmhost::drift_integral(co, a0, a1);
}

Layout plan(const pm_config& c) {
    Layout L;
    const size_t sT = c.precision == PM_FP64 ? 8 : 4, sC = 2 * sT;
    const size_t np3 = (size_t)c.np * c.np * c.np;
    const size_t n = c.nmesh, n3 = n * n * n, nspec = (n / 2 + 1) * n * n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.x = take(3 * np3 * sT);
    L.p = take(3 * np3 * sT);
    L.rho = take(n3 * sT);
    for (int j = 0; j < 3; ++j) L.spec[j] = take(nspec * sC);
    for (int j = 0; j < 3; ++j) L.force[j] = take(n3 * sT);
    L.gr = c.mode == PM_GR_POISSON;
    if (L.gr) L.phi_old = take(nspec * sC);
    L.has_island = L.gr && c.n_lo > 0;
    if (L.has_island) L.island = take((size_t)(c.n_lo + 1) * (2 * c.n_lo + 1) * (2 * c.n_lo + 1) * 16);
    L.amp = take((3 * (size_t)(c.np / 2) * (c.np / 2) + 1) * 8);
    L.bin_of = take((3 * (n / 2) * (n / 2) + 1) * 2);
    L.wtab = take((n / 2 + 1) * 8);
    L.acc = take(2 * kMaxBins * 8);
    L.mid = take(mid_sync_words_count((int)(n / 2 + 1)) * 4);
    L.has_mid = true;
    L.total = off;
    return L;
}

}  // namespace

struct pm_ctx {
    pm_config cfg;
    Layout L;
    unsigned char* ws = nullptr;
    cudaStream_t st = nullptr;
    pmhost::Cosmo cosmo;
    int n = 0, np = 0;
    int64_t np3 = 0;
    double kf = 0.0;
    int step = 0;
    bool synced = true;
    bool have_phi = false;
    double a_last = 0.0;
    // device scratch of the halo-proxy selection (spectrum buffers by default)
    size_t scratch_off = 0, scratch_bytes = 0;
    // rho holds the counting density of the current positions (left by the fused
    // kick-drift-deposit pass of the previous step)
    bool rho_valid = false;
    // when set, the force meshes of the step (three n^3 meshes back to back) live here
    // instead of L.force (the gradient's forward re-run writes them straight into its record)
    void* force_at = nullptr;
    void* force(int j) { return force_at ? (void*)((char*)force_at + (size_t)j * n * n * n * sT()) : at(L.force[j]); }
    // when set, the positions of the step are read from x_at and the fused update writes the
    // drifted ones to x_out (the gradient's re-run records each step's positions this way)
    void* x_at = nullptr;
    void* x_out = nullptr;
    void* xpos() { return x_at ? x_at : at(L.x); }
    // per-phase timing (pm_profile / pm_timings)
    bool prof = false;
    std::vector<cudaEvent_t> pool;
    struct Rec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    cudaEvent_t take_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // second stream of the gradient's overlapped forward re-runs (created on first use)
    cudaStream_t st2 = nullptr;
    // the recorded forward run of the reverse sweep (pm_adjoint_record -> pm_adjoint_run)
    struct AdjSession {
        void* scratch = nullptr;
        size_t bytes = 0;
        int C = 0;
        std::vector<cudaEvent_t> ev_ckpt, ev_rerun, ev_rev;
        bool recorded = false;
        ~AdjSession() {
            for (auto* v : {&ev_ckpt, &ev_rerun, &ev_rev})
                for (auto e : *v) cudaEventDestroy(e);
        }
    };
    AdjSession* adj = nullptr;
    // CTA size of the fused middle passes of the force evaluation (0: the separate passes;
    // pm_set_fused_fft, pm_autotune_fft)
    int mid_threads = 0;
    // integer triangle counts of the last bispectrum geometry (pm_bispectrum)
    struct BkCounts {
        int n = 0, m = 0;
        std::vector<double> edges, counts;
    };
    BkCounts bk_counts;
    ~pm_ctx() {
        delete adj;
        if (st2) cudaStreamDestroy(st2);
        for (auto& r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
    void* at(size_t off) const { return ws + off; }
    double a_grid(int i) const { return cfg.a_init + ((cfg.a_final - cfg.a_init) * i) / cfg.n_steps; }
    bool fp64() const { return cfg.precision == PM_FP64; }
    size_t sT() const { return fp64() ? 8 : 4; }
};

namespace {

// Records a CUDA event pair around one phase when profiling is on.
struct Phase {
    pm_ctx* c;
    int id;
    cudaEvent_t a = nullptr;
    Phase(pm_ctx* ctx, int phase) : c(ctx), id(phase) {
        if (c->prof) {
            a = c->take_event();
            cudaEventRecord(a, c->st);
        }
    }
    ~Phase() {
        if (a) {
            cudaEvent_t b = c->take_event();
            cudaEventRecord(b, c->st);
            c->recs.push_back({id, a, b});
        }
    }
};

// Forward z and y passes of a real mesh of side n into spec, `sub` subtracted from every
// value (kDensityMean for the particle density: its zero mode is dropped by every operator).
template <typename T>
pm_status forward_to_y(pm_ctx* c, const void* real, void* spec, int n, double sub = 0.0) {
    Phase ph(c, PM_PHASE_FFT_ZY_FWD);
    PM_CK(forward_zy<T>((const T*)real, (cplx<T>*)spec, n, 1, c->st, sub));
    return PM_OK;
}

// The three-output gradient chain on the np^3 lattice: out_j = sum_n (-i k_j) F(g_n) e^{i n.q}
// with g the spectrum in spec[0] (real_in == null) or the forward transform of real_in,
// and F the OP_ZA filter of op (Zel'dovich amplitude, identity or inverse Laplacian).
template <typename T>
pm_status za_chain(pm_ctx* c, const void* real_in, SpecOp op, void* const* out) {
    const int np = c->np;
    cplx<T>* s0 = (cplx<T>*)c->at(c->L.spec[0]);
    cplx<T>* s1 = (cplx<T>*)c->at(c->L.spec[1]);
    cplx<T>* s2 = (cplx<T>*)c->at(c->L.spec[2]);
    op.kind = OP_ZA;
    op.kf = c->kf;
    op.fwd = real_in ? 1 : 0;
    if (real_in) PM_TRY(forward_to_y<T>(c, real_in, s0, np));
    PM_CK(x_cols<T>(s0, s1, np / 2 + 1, np, op, c->st));
    PM_CK(y_rows_grad3<T>(s0, s1, s2, (int64_t)(np / 2 + 1) * np, np, c->kf, c->st));
    const cplx<T>* in[3] = {s1, s2, s0};
    T* o[3] = {(T*)out[0], (T*)out[1], (T*)out[2]};
    PM_CK(z_c2r<T>(in, o, 3, np, 1, 4u, c->kf, c->st));
    return PM_OK;
}

// Second-order LPT displacement Psi2 (into out) from Psi1 (three np^3 meshes): the
// derivatives of each Psi1 component build the source S in two scratch meshes, then
// Psi2 = grad phi2 with laplacian(phi2) = S.  Modes with a Nyquist component are dropped,
// as in the first-order displacement.
template <typename T>
pm_status lpt2_displacement(pm_ctx* c, void* const* psi1, void* s, void* a, void* const* out) {
    const double inv_n3 = std::pow((double)c->np, -3.0);
    for (int comp = 0; comp < 3; ++comp) {
        SpecOp od;
        od.za_filter = ZA_IDENTITY;  // out_j = d_j Psi1_comp
        od.coef = -inv_n3;
        od.amp = (const double*)c->at(c->L.amp);
        PM_TRY(za_chain<T>(c, psi1[comp], od, out));
        PM_CK(lpt2_source(comp, out, s, a, c->np3, c->cfg.precision, c->st));
    }
    SpecOp o2;
    o2.za_filter = ZA_INV_LAPLACE;  // out_j = d_j phi2, phi2 = laplacian^-1 S
    o2.coef = inv_n3;
    o2.amp = (const double*)c->at(c->L.amp);
    return za_chain<T>(c, s, o2, out);
}

// Counting density of the context's particles (mass (n/np)^3 per particle) on rho.
pm_status deposit_particles(pm_ctx* c, void* rho) {
    Phase ph(c, PM_PHASE_DEPOSIT);
    PM_CK(cudaMemsetAsync(rho, 0, c->sT() * (size_t)c->n * c->n * c->n, c->st));
    const double mass = std::pow((double)c->n / c->np, 3);
    PM_CK(deposit_lattice(c->xpos(), c->np, c->cfg.precision, c->n, mass, rho, c->st));
    return PM_OK;
}

// rho holding the counting density of the current particles: the one the last fused update
// left there when it is still valid (the positions have not moved since), else a new deposit.
pm_status current_density(pm_ctx* c, const void** rho_out) {
    void* rho = c->at(c->L.rho);
    if (!c->rho_valid) {
        PM_TRY(deposit_particles(c, rho));
        c->rho_valid = true;
    }
    *rho_out = rho;
    return PM_OK;
}

// Force meshes g = -grad phi of the current particles at scale factor a.
bool fused_update(const pm_ctx* c) { return ikd_deposit_supported(c->np, c->cfg.precision, c->n); }
// Forms of the forward y, x and inverse y passes of the spectral force (FP32): 0 = three
// separate launches; 1 = whole kz planes in shared memory (meshes of 64^3 and 128^3);
// 256 / 512 / 1024 = one persistent launch over the planes with CTAs of that size (256^3 and up).
constexpr int kFormPlane = 1;
bool form_applies(int form, const pm_ctx* c) {
    if (c->fp64() || c->cfg.gradient != PM_GRAD_SPECTRAL) return form == 0;
    if (form == kFormPlane) return c->n == 64 || c->n == 128;
    if (form == 256 || form == 512 || form == 1024) return c->n >= 256 && c->L.has_mid;
    return form == 0;
}
bool fused_middle_applies(const pm_ctx* c) { return form_applies(512, c); }
bool fused_middle(const pm_ctx* c) { return c->mid_threads > 1 && form_applies(c->mid_threads, c); }
bool plane_middle(const pm_ctx* c) { return c->mid_threads == kFormPlane && form_applies(kFormPlane, c); }

// The fused middle passes' error word (set when one of their bounded waits gave up; it stays
// set): PM_ERR_TIMEOUT if it is.  Synchronises the context stream.
pm_status check_wait_error(pm_ctx* c) {
    if (!c->L.has_mid) return PM_OK;  // batch views: their passes never wait
    unsigned err = 0;
    const size_t word = mid_sync_words_count(c->n / 2 + 1) - 1;
    PM_CK(cudaMemcpyAsync(&err, (unsigned*)c->at(c->L.mid) + word, sizeof(err), cudaMemcpyDeviceToHost, c->st));
    PM_CK(cudaStreamSynchronize(c->st));
    if (err) return fail(PM_ERR_TIMEOUT, "a bounded device wait of the fused FFT passes gave up; results are invalid");
    return PM_OK;
}

template <typename T>
pm_status compute_forces_t(pm_ctx* c, double a) {
    const int n = c->n;
    void* rho = c->at(c->L.rho);
    if (!c->rho_valid) PM_TRY(deposit_particles(c, rho));
    cplx<T>* s0 = (cplx<T>*)c->at(c->L.spec[0]);
    cplx<T>* s1 = (cplx<T>*)c->at(c->L.spec[1]);
    cplx<T>* s2 = (cplx<T>*)c->at(c->L.spec[2]);
    if (fused_middle(c) || plane_middle(c)) {
        // the forward y pass runs inside the fused or whole-plane middle passes
        Phase ph(c, PM_PHASE_FFT_ZY_FWD);
        PM_CK(z_r2c<T>((const T*)rho, s0, n, 1, c->st, kDensityMean));
    } else {
        PM_TRY(forward_to_y<T>(c, rho, s0, n, kDensityMean));
    }
    // the forward z pass has consumed rho: the fused update deposits the next density there, so
    // the inverse z pass clears it beside the force rows it writes (every form of the passes)
    T* clear = fused_update(c) ? (T*)rho : nullptr;
    c->rho_valid = false;
    SpecOp op;
    op.kf = c->kf;
    op.fwd = 1;
    const double n3 = (double)n * n * n;
    if (c->cfg.mode == PM_NEWTON) {
        op.kind = OP_NEWTON;
        op.coef = -1.5 * c->cfg.omega_m / n3;
    } else {
        op.kind = OP_GR;
        op.calH = pmhost::conformal_hubble(c->cosmo, a);
        op.omm_a = pmhost::omega_m_a(c->cosmo, a);
        op.first = c->have_phi ? 0 : 1;
        op.inv_dtau = c->have_phi ? 1.0 / (pmhost::kCLight * pmhost::kick_integral(c->cosmo, c->a_last, a)) : 0.0;
        op.ac2_over_n3 = a * pmhost::kCLight * pmhost::kCLight / n3;
        op.n_lo = c->L.has_island ? c->cfg.n_lo : 0;
        op.phi_old = c->at(c->L.phi_old);
        op.island = c->L.has_island ? (double2*)c->at(c->L.island) : nullptr;
    }
    if (c->cfg.gradient == PM_GRAD_FD1) {
        // the potential alone goes back to real space (force(0)); the update differentiates
        // its CIC interpolant (the Poisson-gauge pass still writes its x gradient, unused)
        if (op.kind == OP_NEWTON) op.kind = OP_POTENTIAL;
        {
            Phase ph(c, PM_PHASE_FFT_X_GREEN);
            PM_CK(x_cols<T>(s0, op.kind == OP_POTENTIAL ? nullptr : s1, n / 2 + 1, n, op, c->st));
        }
        Phase ph(c, PM_PHASE_FFT_YZ_INV);
        PM_CK((y_rows<T, true>(s0, (int64_t)(n / 2 + 1) * n, n, c->st)));
        const cplx<T>* in[1] = {s0};
        T* out[1] = {(T*)c->force(0)};
        PM_CK(z_c2r<T>(in, out, 1, n, 1, 0u, 0.0, c->st, nullptr, clear));
    } else if (plane_middle(c)) {
        {
            Phase ph(c, PM_PHASE_FFT_X_GREEN);
            PM_CK(fft_plane<T>(s0, s1, s2, n / 2 + 1, n, op, c->st));
        }
        Phase ph(c, PM_PHASE_FFT_YZ_INV);
        const cplx<T>* in[3] = {s1, s2, s0};  // -i k_j phi back along x and y, j = x, y, z
        T* out[3] = {(T*)c->force(0), (T*)c->force(1), (T*)c->force(2)};
        PM_CK(z_c2r<T>(in, out, 3, n, 1, 0u, c->kf, c->st, nullptr, clear));
    } else if (fused_middle(c)) {
        // z r2c above left the half spectrum in s0 before its forward y pass (see forward_to_y)
        {
            Phase ph(c, PM_PHASE_FFT_X_GREEN);
            PM_CK(fft_middle<T>(s0, s1, s2, n / 2 + 1, n, op, (unsigned*)c->at(c->L.mid), c->mid_threads, c->st));
        }
        Phase ph(c, PM_PHASE_FFT_YZ_INV);
        const cplx<T>* in[3] = {s1, s2, s0};  // IFFT_y(-i kx phi), IFFT_y(-i ky phi), IFFT_y(phi) (-i kz)
        T* out[3] = {(T*)c->force(0), (T*)c->force(1), (T*)c->force(2)};
        PM_CK(z_c2r<T>(in, out, 3, n, 1, 4u, c->kf, c->st, nullptr, clear));
    } else {
        {
            Phase ph(c, PM_PHASE_FFT_X_GREEN);
            PM_CK(x_cols<T>(s0, s1, n / 2 + 1, n, op, c->st));
        }
        Phase ph(c, PM_PHASE_FFT_YZ_INV);
        T* out[3] = {(T*)c->force(0), (T*)c->force(1), (T*)c->force(2)};
        PM_CK(inverse_yz_grad<T>(s0, s1, s2, out, n, 1, c->kf, c->st, nullptr, clear));
    }
    if (c->cfg.mode == PM_GR_POISSON) {
        c->have_phi = true;
        c->a_last = a;
    }
    return PM_OK;
}

pm_status compute_forces(pm_ctx* c, double a) {
    return c->fp64() ? compute_forces_t<double>(c, a) : compute_forces_t<float>(c, a);
}

pm_status kick_drift(pm_ctx* c, double kick, double drift) {
    Phase ph(c, PM_PHASE_KICK_DRIFT);
    void* g[3] = {c->force(0), c->force(1), c->force(2)};
    // first-order gradient: force(0) holds the potential, differentiated across the cell of spacing L/n
    const double fd_inv_d = c->cfg.gradient == PM_GRAD_FD1 ? c->n / c->cfg.box : 0.0;
    if (fused_update(c)) {
        PM_CK(interp_kick_drift_deposit(c->xpos(), c->at(c->L.p), c->np, c->cfg.precision, c->n, g, kick, drift,
                                        c->cfg.box, std::pow((double)c->n / c->np, 3), c->at(c->L.rho), c->st, 1,
                                        nullptr, c->x_out, fd_inv_d));
        c->rho_valid = true;
        return PM_OK;
    }
    if (c->x_at || c->x_out) return fail(PM_ERR_UNSUPPORTED, "out-of-place positions need the fused update");
    PM_CK(interp_kick_drift(c->at(c->L.x), c->at(c->L.p), c->np3, c->cfg.precision, c->n, g, kick, drift,
                            c->cfg.box, c->st, fd_inv_d));
    return PM_OK;
}

// Bin table of the context mesh on the device (every |n|^2 <= 3 (n/2)^2), built by a kernel
// from the squared edges staged in the context's accumulator area; the host keeps the same
// table for |n|^2 <= (n/2)^2 (the binned modes) in host_tab, from the same comparisons.
pm_status upload_bin_table(pm_ctx* c, int nbins, const double* edges, std::vector<int16_t>& host_tab) {
    const int n = c->n;
    std::vector<double> e2(nbins + 1);
    for (int b = 0; b <= nbins; ++b) e2[b] = edges[b] * edges[b];
    double* e2_dev = (double*)c->at(c->L.acc);
    PM_CK(cudaMemcpyAsync(e2_dev, e2.data(), sizeof(double) * (nbins + 1), cudaMemcpyHostToDevice, c->st));
    PM_CK(bin_table((int16_t*)c->at(c->L.bin_of), 3 * (int64_t)(n / 2) * (n / 2), e2_dev, nbins, c->st));
    const int64_t top = (int64_t)(n / 2) * (n / 2);
    host_tab.assign(top + 1, (int16_t)-1);
    int q = -1;  // largest edge index with e2[q] <= s, advanced as s grows
    for (int64_t s = 0; s <= top; ++s) {
        const double v = (double)s;
        while (q < nbins && e2[q + 1] <= v) ++q;
        int b = q;
        if (v == e2[nbins]) b = nbins - 1;
        host_tab[s] = (b >= 0 && b < nbins) ? (int16_t)b : (int16_t)-1;
    }
    return PM_OK;
}

// Weighted number of modes with |n|^2 = s for s <= (n/2)^2 over the stored half spectrum
// (kx, ky in [-n/2, n/2), kz in [0, n/2]): weight 1 on the kz = 0 and n/2 planes and 2
// elsewhere, which counts the mirrored half.  Geometry only, so one table per mesh size.
const std::vector<double>& mode_counts(int n) {
    static std::mutex mu;
    static std::map<int, std::vector<double>> cache;
    std::lock_guard<std::mutex> g(mu);
    const auto it = cache.find(n);
    if (it != cache.end()) return it->second;
    const int64_t M = n / 2, top = M * M;
    std::vector<double> c2(top + 1, 0.0);  // (kx, ky) pairs with kx^2 + ky^2 = s
    for (int64_t a = -M; a < M; ++a)
        for (int64_t b = -M; b < M; ++b)
            if (a * a + b * b <= top) c2[a * a + b * b] += 1.0;
    std::vector<double> cnt(top + 1, 0.0);
    for (int64_t z = 0; z <= M; ++z) {
        const double w = (z == 0 || z == M) ? 1.0 : 2.0;
        for (int64_t s = 0; s + z * z <= top; ++s) cnt[s + z * z] += w * c2[s];
    }
    return cache.emplace(n, std::move(cnt)).first->second;
}

pm_status check_edges(int nbins, const double* edges) {
    if (nbins < 1 || nbins > kMaxBins || !edges) return fail(PM_ERR_INVALID_ARG, "need 1..256 bins and edges");
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b] >= 0 && edges[b + 1] > edges[b])) return fail(PM_ERR_INVALID_ARG, "edges must increase");
    return PM_OK;
}

// p2_out (with field2 only): the auto spectrum of field2 from the same pass.
template <typename T>
pm_status power_t(pm_ctx* c, const void* field, const void* field2, int nbins, const double* edges, int deconv,
                  double* k_out, double* p_out, double* nmodes_out, double* p2_out = nullptr) {
    const int n = c->n;
    const void* f1 = field;
    if (!f1) PM_TRY(current_density(c, &f1));
    void* s0 = c->at(c->L.spec[0]);
    void* s1 = c->at(c->L.spec[1]);
    PM_TRY(forward_to_y<T>(c, f1, s0, n, field ? 0.0 : kDensityMean));
    if (field2) PM_TRY(forward_to_y<T>(c, field2, s1, n));
    std::vector<int16_t> tab;
    PM_TRY(upload_bin_table(c, nbins, edges, tab));
    // per-CTA rows of bin sums in the third spectrum buffer (free here), reduced in a fixed order
    const bool two = field2 && p2_out;
    double* rows = (double*)c->at(c->L.spec[2]);
    const size_t spec_bytes = (size_t)(n / 2 + 1) * n * n * 2 * c->sT();
    const int nrows = (int)std::min<size_t>(4 * (size_t)num_sms(), spec_bytes / (sizeof(double) * nbins * (two ? 2 : 1)));
    double* rows2 = two ? rows + (size_t)nrows * nbins : nullptr;
    PM_CK(cudaMemsetAsync(rows, 0, sizeof(double) * nrows * nbins * (two ? 2 : 1), c->st));
    SpecOp op;
    op.kind = OP_BIN;
    op.fwd = 1;
    op.kf = c->kf;
    op.bin_of = (const int16_t*)c->at(c->L.bin_of);
    op.wtab = (const double*)c->at(c->L.wtab);
    op.acc = rows;
    op.acc2 = rows2;
    op.acc_rows = nrows;
    op.nbins = nbins;
    op.deconv = deconv ? 1 : 0;
    op.in2 = field2 ? s1 : nullptr;
    PM_CK(x_cols<T>((cplx<T>*)s0, nullptr, n / 2 + 1, n, op, c->st));
    double* acc = (double*)c->at(c->L.acc);
    PM_CK(bin_rows_sum(rows, nrows, nbins, acc, c->st));
    if (two) PM_CK(bin_rows_sum(rows2, nrows, nbins, acc + nbins, c->st));
    // mode counts and mean |k| per bin follow from the geometry alone: summed on the host while
    // the device transforms and bins (the copy below waits for it)
    const std::vector<double>& cnt = mode_counts(n);
    std::vector<double> nm(nbins, 0.0), ks(nbins, 0.0);
    for (size_t s = 1; s < cnt.size(); ++s) {
        const int b = tab[s];
        if (b < 0) continue;
        nm[b] += cnt[s];
        ks[b] += cnt[s] * std::sqrt((double)s);
    }
    std::vector<double> h((two ? 2 : 1) * nbins);
    PM_CK(cudaMemcpyAsync(h.data(), acc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st));
    PM_CK(cudaStreamSynchronize(c->st));
    const double V = c->cfg.box * c->cfg.box * c->cfg.box;
    const double n6 = std::pow((double)n, 6);
    for (int b = 0; b < nbins; ++b) {
        const double w = nm[b];
        if (nmodes_out) nmodes_out[b] = w;
        if (w > 0) {
            if (p_out) p_out[b] = V / n6 * h[b] / w;
            if (k_out) k_out[b] = c->kf * ks[b] / w;
            if (two) p2_out[b] = V / n6 * h[nbins + b] / w;
        } else {
            if (p_out) p_out[b] = NAN;
            if (k_out) k_out[b] = NAN;
            if (two) p2_out[b] = NAN;
        }
    }
    return PM_OK;
}

struct BkLayout {
    size_t specs, fields, tri, accS, accC, total;
    int ntri;
};
BkLayout bk_plan(int sT, int m, int nbins) {
    BkLayout B;
    const size_t per_spec = (size_t)(m / 2 + 1) * m * m * 2 * sT;
    const size_t per_field = (size_t)m * m * m * sT;
    B.ntri = nbins * (nbins + 1) * (nbins + 2) / 6;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    B.specs = take(2 * (size_t)nbins * per_spec);
    B.fields = take(2 * (size_t)nbins * per_field);
    B.tri = take(sizeof(int4) * (size_t)B.ntri);
    B.accS = take(sizeof(double) * (size_t)B.ntri);
    B.accC = take(sizeof(double) * (size_t)B.ntri);
    B.total = off;
    return B;
}

// Integer triangle counts N_ijl of the bin triplets on the m grid for an n^3 field, cached per
// (n, m, edges): the FFT identity on the indicator fields, run in FP64 (the FP32 sums of counts of
// 1e6 - 1e7 configurations are off by units) in the scratch's spectrum and field areas, which
// hold nbins FP64 spectra and fields in either precision.
pm_status bk_counts(pm_ctx* c, int nbins, const double* edges, int m, unsigned char* scratch, const BkLayout& B,
                    const int4* dunits, int nunits, const std::vector<double>** out) {
    pm_ctx::BkCounts& K = c->bk_counts;
    const std::vector<double> e(edges, edges + nbins + 1);
    if (!(K.n == c->n && K.m == m && K.edges == e)) {
        double2* specs = (double2*)(scratch + B.specs);
        double* fields = (double*)(scratch + B.fields);
        double* acc = (double*)(scratch + B.accC);
        PM_CK(bk_indicators(c->n, specs, m, nbins, (const int16_t*)c->at(c->L.bin_of), c->st));
        SpecOp inv;
        inv.kind = OP_INV;
        inv.fwd = 0;
        PM_CK(x_cols<double>(specs, nullptr, nbins * (m / 2 + 1), m, inv, c->st));
        PM_CK((y_rows<double, true>(specs, (int64_t)nbins * (m / 2 + 1) * m, m, c->st)));
        const double2* in[1] = {specs};
        double* o[1] = {fields};
        PM_CK(z_c2r<double>(in, o, 1, m, nbins, 0u, 0.0, c->st));
        PM_CK(cudaMemsetAsync(acc, 0, sizeof(double) * B.ntri, c->st));
        PM_CK(bk_units<double>(fields, m, nbins, dunits, nunits, acc, c->st));
        std::vector<double> hc(B.ntri);
        PM_CK(cudaMemcpyAsync(hc.data(), acc, sizeof(double) * B.ntri, cudaMemcpyDeviceToHost, c->st));
        PM_CK(cudaStreamSynchronize(c->st));
        const double m3 = (double)m * m * m;
        K.counts.resize(B.ntri);
        for (int t = 0; t < B.ntri; ++t) K.counts[t] = std::rint(hc[t] / m3);
        K.n = c->n;
        K.m = m;
        K.edges = e;
    }
    *out = &K.counts;
    return PM_OK;
}

template <typename T>
pm_status bispectrum_t(pm_ctx* c, const void* field, int nbins, const double* edges, int m, int deconv,
                       unsigned char* scratch, const BkLayout& B, double* b_out, double* ntri_out) {
    const int n = c->n;
    const void* f1 = field;
    if (!f1) PM_TRY(current_density(c, &f1));
    std::vector<int16_t> tab;
    PM_TRY(upload_bin_table(c, nbins, edges, tab));
    // units (i, j-block of 4, l-block of 8) with at least one triangle i <= j <= l (see bk_units):
    // every block from the one holding j = i on, and l-blocks from the one holding its first j;
    // never more units than triangles
    std::vector<int4> units;
    units.reserve(B.ntri);
    for (int i = 0, t = 0; i < nbins; ++i) {
        const int Ti = t;  // index of triangle (i, i, i)
        for (int j = i; j < nbins; ++j) t += nbins - j;
        for (int jb = i / 4; 4 * jb < nbins; ++jb)
            for (int lb = jb / 2; 8 * lb < nbins; ++lb) units.push_back(make_int4(i, jb, lb, Ti));
    }
    int4* dunits = (int4*)(scratch + B.tri);
    PM_CK(cudaMemcpyAsync(dunits, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice, c->st));
    const std::vector<double>* counts = nullptr;
    PM_TRY(bk_counts(c, nbins, edges, m, scratch, B, dunits, (int)units.size(), &counts));
    // the data: forward transform of the field, masked spectra on the m grid, their inverse
    // transforms, the triple-product sums
    cplx<T>* s0 = (cplx<T>*)c->at(c->L.spec[0]);
    PM_TRY(forward_to_y<T>(c, f1, s0, n, field ? 0.0 : kDensityMean));
    SpecOp fw;
    fw.kind = OP_FWD_STORE;
    fw.fwd = 1;
    PM_CK(x_cols<T>(s0, nullptr, n / 2 + 1, n, fw, c->st));
    cplx<T>* specs = (cplx<T>*)(scratch + B.specs);
    T* fields = (T*)(scratch + B.fields);
    PM_CK(bk_masks<T>(s0, n, specs, m, nbins, (const int16_t*)c->at(c->L.bin_of), (const double*)c->at(c->L.wtab),
                      deconv ? 1 : 0, c->st));
    SpecOp inv;
    inv.kind = OP_INV;
    inv.fwd = 0;
    PM_CK(x_cols<T>(specs, nullptr, nbins * (m / 2 + 1), m, inv, c->st));
    PM_CK((y_rows<T, true>(specs, (int64_t)nbins * (m / 2 + 1) * m, m, c->st)));
    const cplx<T>* in[1] = {specs};
    T* out[1] = {fields};
    PM_CK(z_c2r<T>(in, out, 1, m, nbins, 0u, 0.0, c->st));
    double* accS = (double*)(scratch + B.accS);
    PM_CK(cudaMemsetAsync(accS, 0, sizeof(double) * B.ntri, c->st));
    PM_CK(bk_units<T>(fields, m, nbins, dunits, (int)units.size(), accS, c->st));
    std::vector<double> hs(B.ntri);
    PM_CK(cudaMemcpyAsync(hs.data(), accS, sizeof(double) * B.ntri, cudaMemcpyDeviceToHost, c->st));
    PM_CK(cudaStreamSynchronize(c->st));
    const double V = c->cfg.box * c->cfg.box * c->cfg.box;
    const double n9 = std::pow((double)n, 9);
    const double m3 = (double)m * m * m;
    // B divides the triangle sum by the exact integer count of configurations
    for (int t = 0; t < B.ntri; ++t) {
        const double cnt = (*counts)[t];
        if (ntri_out) ntri_out[t] = cnt;
        if (b_out) b_out[t] = (cnt > 0.0) ? V * V / n9 * (hs[t] / m3) / cnt : NAN;
    }
    return PM_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* pm_version(void) { return "pm-gb300 0.2 (sm_103a)"; }

const char* pm_last_error(void) { return g_err.c_str(); }

pm_status pm_step_factors(const pm_config* cfg, int s, double* kick, double* drift, double* kick_close) {
    PM_TRY(validate(cfg));
    if (s < 0 || s >= cfg->n_steps) return fail(PM_ERR_INVALID_ARG, "step outside 0..n_steps-1");
    pmhost::Cosmo co;
    co.omega_m = cfg->omega_m;
    co.omega_b = cfg->omega_b;
    co.h = cfg->h;
    co.n_s = cfg->n_s;
    co.sigma8 = cfg->sigma8;
    auto grid = [cfg](int i) { return cfg->a_init + ((cfg->a_final - cfg->a_init) * i) / cfg->n_steps; };
    const double a0 = grid(s), a1 = grid(s + 1), ah = 0.5 * (a0 + a1);
    const double a_from = (s == 0) ? a0 : 0.5 * (grid(s - 1) + a0);
    if (kick) *kick = kick_factor(*cfg, co, a_from, ah, a0);
    if (drift) *drift = drift_factor(*cfg, co, a0, a1, ah);
    const int N = cfg->n_steps;
    if (kick_close) *kick_close = kick_factor(*cfg, co, 0.5 * (grid(N - 1) + grid(N)), grid(N), grid(N));
    return PM_OK;
}

pm_status pm_linear_power(const pm_config* cfg, double a, const double* k, int64_t count, double* p_out,
                          double* D_out, double* f_out) {
    if (!cfg || count < 0 || (count > 0 && (!k || !p_out))) return fail(PM_ERR_INVALID_ARG, "bad arguments");
    if (!(cfg->omega_m > 0 && cfg->omega_m <= 1) || !(a > 0)) return fail(PM_ERR_INVALID_ARG, "bad omega_m or a");
    for (int64_t i = 0; i < count; ++i)
        if (!(k[i] >= 0)) return fail(PM_ERR_INVALID_ARG, "k must be non-negative");
    pmhost::Cosmo co;
    co.omega_m = cfg->omega_m;
    co.omega_b = cfg->omega_b;
    co.h = cfg->h;
    co.n_s = cfg->n_s;
    co.sigma8 = cfg->sigma8;
    pmhost::normalise_sigma8(co);
    const double D = pmhost::growth_D(co, a);
    for (int64_t i = 0; i < count; ++i) p_out[i] = k[i] > 0 ? pmhost::power_linear(co, k[i]) * D * D : 0.0;
    if (D_out) *D_out = D;
    if (f_out) *f_out = pmhost::growth_f(co, a);
    return PM_OK;
}

pm_status pm_b1_gr_theory(const pm_config* cfg, double a, double b1, double* b1_gr) {
    if (!cfg || !b1_gr) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (!(cfg->omega_m > 0 && cfg->omega_m <= 1) || !(a > 0)) return fail(PM_ERR_INVALID_ARG, "bad omega_m or a");
    pmhost::Cosmo cosmo;
    cosmo.omega_m = cfg->omega_m;
    cosmo.omega_b = cfg->omega_b;
    cosmo.h = cfg->h;
    cosmo.n_s = cfg->n_s;
    cosmo.sigma8 = cfg->sigma8;
    // Eq. bgr: b1^GR = 3 (f + (3/2) Omega_m(a)) (1 - b1)
    *b1_gr = 3.0 * (pmhost::growth_f(cosmo, a) + 1.5 * pmhost::omega_m_a(cosmo, a)) * (1.0 - b1);
    return PM_OK;
}

pm_status pm_workspace_size(const pm_config* cfg, size_t* bytes) {
    PM_TRY(validate(cfg));
    if (!bytes) return fail(PM_ERR_INVALID_ARG, "null bytes");
    *bytes = plan(*cfg).total;
    return PM_OK;
}

pm_status pm_init(const pm_config* cfg, void* workspace, size_t bytes, void* stream, pm_ctx** out) {
    PM_TRY(validate(cfg));
    if (!out) return fail(PM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    const Layout L = plan(*cfg);
    if (!workspace || bytes < L.total) return fail(PM_ERR_WORKSPACE, "workspace smaller than pm_workspace_size");
    if ((uintptr_t)workspace % 256) return fail(PM_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    PM_TRY(check_device());
    pm_ctx* c = new pm_ctx();
    c->cfg = *cfg;
    c->L = L;
    c->ws = (unsigned char*)workspace;
    c->st = (cudaStream_t)stream;
    c->n = cfg->nmesh;
    c->np = cfg->np;
    c->np3 = (int64_t)cfg->np * cfg->np * cfg->np;
    c->kf = 2.0 * M_PI / cfg->box;
    c->scratch_off = L.spec[0];
    c->scratch_bytes = L.force[0] - L.spec[0];
    c->cosmo.omega_m = cfg->omega_m;
    c->cosmo.omega_b = cfg->omega_b;
    c->cosmo.h = cfg->h;
    c->cosmo.n_s = cfg->n_s;
    c->cosmo.sigma8 = cfg->sigma8;
    pmhost::normalise_sigma8(c->cosmo);
    // sqrt(P(k)/V) per integer |n|^2 on the particle lattice, and the CIC window per |n_j|
    const int hp = cfg->np / 2;
    std::vector<double> amp(3 * (size_t)hp * hp + 1, 0.0);
    const double V = cfg->box * cfg->box * cfg->box;
    for (size_t n2 = 1; n2 < amp.size(); ++n2)
        amp[n2] = std::sqrt(pmhost::power_linear(c->cosmo, c->kf * std::sqrt((double)n2)) / V);
    std::vector<double> wtab(c->n / 2 + 1);
    for (int mq = 0; mq <= c->n / 2; ++mq) {
        const double x = M_PI * mq / c->n;
        const double s = (mq == 0) ? 1.0 : std::sin(x) / x;
        wtab[mq] = s * s;
    }
    cudaError_t e = cudaMemcpyAsync(c->at(L.amp), amp.data(), amp.size() * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->at(L.wtab), wtab.data(), wtab.size() * 8, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->at(L.mid), 0, mid_sync_words_count(c->n / 2 + 1) * 4, c->st);
    if (e == cudaSuccess && L.has_island)
        e = cudaMemsetAsync(c->at(L.island), 0, (size_t)(cfg->n_lo + 1) * (2 * cfg->n_lo + 1) * (2 * cfg->n_lo + 1) * 16,
                            c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        delete c;
        return fail(PM_ERR_CUDA, std::string("pm_init: ") + cudaGetErrorString(e));
    }
    *out = c;
    return PM_OK;
}

pm_status pm_destroy(pm_ctx* ctx) {
    delete ctx;
    return PM_OK;
}

pm_status pm_particles(pm_ctx* c, void** x, void** p) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (x) *x = c->at(c->L.x);
    if (p) *p = c->at(c->L.p);
    return PM_OK;
}

}  // extern "C"

namespace {

// FP64 positions are box fractions: every one must be finite and in [0, 1) before it
// reaches the CIC index arithmetic (uint32 ticks are valid by construction).  Counted on
// the device into the context's accumulator area; synchronises the context stream.
pm_status check_positions(pm_ctx* c, const void* x) {
    if (!c->fp64()) return PM_OK;
    unsigned long long* bad = (unsigned long long*)c->at(c->L.acc);
    unsigned long long h = 0;
    PM_CK(count_outside_box((const double*)x, 3 * c->np3, bad, c->st));
    PM_CK(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    PM_CK(cudaStreamSynchronize(c->st));
    if (h) return fail(PM_ERR_BOUNDS, std::to_string(h) + " FP64 positions are not finite or outside [0, 1) box units");
    return PM_OK;
}

pm_status copy_state(pm_ctx* c, const void* x, const void* p, int step, bool synced) {
    PM_TRY(check_positions(c, x));
    if (c->adj) c->adj->recorded = false;
    const size_t bytes = 3 * (size_t)c->np3 * c->sT();
    // the context's own arrays (pm_particles), already written by the caller, are not copied
    if (x != c->at(c->L.x)) PM_CK(cudaMemcpyAsync(c->at(c->L.x), x, bytes, cudaMemcpyDeviceToDevice, c->st));
    if (p != c->at(c->L.p)) PM_CK(cudaMemcpyAsync(c->at(c->L.p), p, bytes, cudaMemcpyDeviceToDevice, c->st));
    c->step = step;
    c->synced = synced;
    c->have_phi = false;
    c->rho_valid = false;
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_set_particles(pm_ctx* c, const void* x, const void* p) {
    if (!c || !x || !p) return fail(PM_ERR_INVALID_ARG, "null argument");
    return copy_state(c, x, p, 0, true);
}

pm_status pm_set_state(pm_ctx* c, const void* x, const void* p, int step, int synchronised) {
    if (!c || !x || !p) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (step < 0 || step > c->cfg.n_steps) return fail(PM_ERR_INVALID_ARG, "step outside 0..n_steps");
    if ((step == 0 || step == c->cfg.n_steps) && !synchronised)
        return fail(PM_ERR_INVALID_ARG, "the momenta are synchronised at the ends of the a-grid");
    if (c->cfg.mode == PM_GR_POISSON && step > 0)
        return fail(PM_ERR_UNSUPPORTED, "a Poisson-gauge run resumes only at step 0 (its Phi history is not restored)");
    return copy_state(c, x, p, step, synchronised != 0);
}

pm_status pm_gr_history(pm_ctx* c, void** phi_old, size_t* phi_bytes, void** island, size_t* island_bytes) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (c->cfg.mode != PM_GR_POISSON) return fail(PM_ERR_UNSUPPORTED, "only a Poisson-gauge context has a Phi history");
    const size_t nspec = (size_t)(c->n / 2 + 1) * c->n * c->n;
    const size_t isl = c->L.has_island ? (size_t)(c->cfg.n_lo + 1) * (2 * c->cfg.n_lo + 1) * (2 * c->cfg.n_lo + 1) * 16 : 0;
    if (phi_old) *phi_old = c->at(c->L.phi_old);
    if (phi_bytes) *phi_bytes = nspec * 2 * c->sT();
    if (island) *island = isl ? c->at(c->L.island) : nullptr;
    if (island_bytes) *island_bytes = isl;
    return PM_OK;
}

pm_status pm_set_state_gr(pm_ctx* c, const void* x, const void* p, int step, int synchronised, const void* phi_old,
                          const void* island) {
    if (!c || !x || !p) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (c->cfg.mode != PM_GR_POISSON) return fail(PM_ERR_INVALID_ARG, "pm_set_state_gr needs a Poisson-gauge context");
    if (step < 0 || step > c->cfg.n_steps) return fail(PM_ERR_INVALID_ARG, "step outside 0..n_steps");
    if ((step == 0 || step == c->cfg.n_steps) && !synchronised)
        return fail(PM_ERR_INVALID_ARG, "the momenta are synchronised at the ends of the a-grid");
    if (step > 0 && (!phi_old || (c->L.has_island && !island)))
        return fail(PM_ERR_INVALID_ARG, "a resumed Poisson-gauge run needs its Phi history (and island)");
    PM_TRY(copy_state(c, x, p, step, synchronised != 0));
    if (step > 0) {
        void* ph = nullptr;
        void* is = nullptr;
        size_t pb = 0, ib = 0;
        PM_TRY(pm_gr_history(c, &ph, &pb, &is, &ib));
        PM_CK(cudaMemcpyAsync(ph, phi_old, pb, cudaMemcpyDeviceToDevice, c->st));
        if (ib) PM_CK(cudaMemcpyAsync(is, island, ib, cudaMemcpyDeviceToDevice, c->st));
        // the last force evaluation: a_{step-1} between steps, a_final after the closing kick
        c->have_phi = true;
        c->a_last = step < c->cfg.n_steps ? c->a_grid(step - 1) : c->a_grid(step);
    }
    return PM_OK;
}

pm_status pm_displacement(pm_ctx* c, void* disp) {
    if (!c || !disp) return fail(PM_ERR_INVALID_ARG, "null argument");
    PM_CK(lagrangian_displacement(c->at(c->L.x), disp, c->np, c->cfg.precision, c->cfg.box, c->st));
    return PM_OK;
}

pm_status pm_positions(pm_ctx* c, void* out) {
    if (!c || !out) return fail(PM_ERR_INVALID_ARG, "null argument");
    PM_CK(positions_mpc(c->at(c->L.x), out, c->np3, c->cfg.precision, c->cfg.box, c->st));
    return PM_OK;
}

pm_status pm_state(pm_ctx* c, int* step, double* a, int* synchronised) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (step) *step = c->step;
    if (a) *a = c->a_grid(c->step);
    if (synchronised) *synchronised = c->synced ? 1 : 0;
    return PM_OK;
}

pm_status pm_ic_zeldovich(pm_ctx* c, uint64_t seed, const void* white_noise, int flags) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (flags & ~(PM_IC_PAIRED | PM_IC_FIXED | PM_IC_2LPT)) return fail(PM_ERR_INVALID_ARG, "unknown IC flags");
    const bool paired = (flags & PM_IC_PAIRED) != 0;
    const int np = c->np;
    const double a = c->cfg.a_init;
    const double D = pmhost::growth_D(c->cosmo, a);
    const double f = pmhost::growth_f(c->cosmo, a);
    const double E = pmhost::E(c->cosmo, a);
    SpecOp op;
    op.za_filter = ZA_AMP;
    op.amp = (const double*)c->at(c->L.amp);
    op.fixed_amp = (flags & PM_IC_FIXED) ? 1 : 0;
    const double sign = paired ? -1.0 : 1.0;
    double scale = 1.0;
    if (white_noise) {
        if (!op.fixed_amp) scale = std::pow((double)np, -1.5);
    } else {
        void* s0 = c->at(c->L.spec[0]);
        if (c->fp64()) PM_CK(noise<double>((double2*)s0, np, seed, c->st));
        else PM_CK(noise<float>((float2*)s0, np, seed, c->st));
    }
    op.coef = -sign * scale;
    void* force[3] = {c->at(c->L.force[0]), c->at(c->L.force[1]), c->at(c->L.force[2])};
    if (!(flags & PM_IC_2LPT)) {
        if (c->fp64()) PM_TRY(za_chain<double>(c, white_noise, op, force));
        else PM_TRY(za_chain<float>(c, white_noise, op, force));
        PM_CK(ic_place(c->at(c->L.x), c->at(c->L.p), force, np, c->cfg.precision, D, a * a * E * f * D, c->cfg.box,
                       c->st));
    } else {
        // Psi1 in the momentum array, the source and its partial sum in the position array
        // (both are written last, by the placement), Psi2 in the force meshes
        const size_t sT = c->sT();
        char* pb = (char*)c->at(c->L.p);
        char* xb = (char*)c->at(c->L.x);
        void* psi1[3] = {pb, pb + c->np3 * sT, pb + 2 * c->np3 * sT};
        void* s = xb;
        void* acc = xb + c->np3 * sT;
        if (c->fp64()) {
            PM_TRY(za_chain<double>(c, white_noise, op, psi1));
            PM_TRY(lpt2_displacement<double>(c, psi1, s, acc, force));
        } else {
            PM_TRY(za_chain<float>(c, white_noise, op, psi1));
            PM_TRY(lpt2_displacement<float>(c, psi1, s, acc, force));
        }
        // second-order growth, D2 = -(3/7) D^2 Om(a)^(-1/143), f2 = 2 Om(a)^(6/11) (Bouchet et al. 1995)
        const double om = pmhost::omega_m_a(c->cosmo, a);
        const double D2 = -3.0 / 7.0 * D * D * std::pow(om, -1.0 / 143.0);
        const double f2 = 2.0 * std::pow(om, 6.0 / 11.0);
        PM_CK(ic_place2(c->at(c->L.x), c->at(c->L.p), psi1, force, np, c->cfg.precision, D, D2, a * a * E * f * D,
                        a * a * E * f2 * D2, c->cfg.box, c->st));
    }
    c->step = 0;
    c->synced = true;
    c->have_phi = false;
    c->rho_valid = false;
    if (c->adj) c->adj->recorded = false;
    return PM_OK;
}

pm_status pm_step(pm_ctx* c, int n_steps) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (n_steps < 0) return fail(PM_ERR_INVALID_ARG, "negative step count");
    if (c->step + n_steps > c->cfg.n_steps) return fail(PM_ERR_STATE, "stepping past a_final");
    for (int k = 0; k < n_steps; ++k) {
        const double a0 = c->a_grid(c->step), a1 = c->a_grid(c->step + 1);
        const double ah = 0.5 * (a0 + a1);
        PM_TRY(compute_forces(c, a0));
        const double a_from = c->synced ? a0 : 0.5 * (c->a_grid(c->step - 1) + a0);
        PM_TRY(kick_drift(c, kick_factor(c->cfg, c->cosmo, a_from, ah, a0), drift_factor(c->cfg, c->cosmo, a0, a1, ah)));
        c->step += 1;
        c->synced = false;
        if (c->step == c->cfg.n_steps) {
            PM_TRY(compute_forces(c, a1));
            PM_TRY(kick_drift(c, kick_factor(c->cfg, c->cosmo, ah, a1, a1), 0.0));
            c->synced = true;
        }
    }
    return PM_OK;
}

pm_status pm_set_fused_fft(pm_ctx* c, int form) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (form != 0 && form != kFormPlane && form != 256 && form != 512 && form != 1024)
        return fail(PM_ERR_INVALID_ARG, "form must be 0 (separate passes), 1 (whole planes), 256, 512 or 1024");
    c->mid_threads = form;
    return PM_OK;
}

pm_status pm_autotune_fft(pm_ctx* c, int* threads_out, double* ms_out) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    if (threads_out) *threads_out = 0;
    if (ms_out) *ms_out = 0.0;
    std::vector<int> cand = {0};
    for (int f : {kFormPlane, 256, 512, 1024})
        if (form_applies(f, c)) cand.push_back(f);
    if (cand.size() == 1) {
        c->mid_threads = 0;
        return PM_OK;
    }
    // the candidates run on the context's spectrum buffers (scratch between force evaluations)
    // with the Newtonian operator, which touches no other state
    const int n = c->n;
    float2* s0 = (float2*)c->at(c->L.spec[0]);
    float2* s1 = (float2*)c->at(c->L.spec[1]);
    float2* s2 = (float2*)c->at(c->L.spec[2]);
    SpecOp op;
    op.kind = OP_NEWTON;
    op.fwd = 1;
    op.kf = c->kf;
    op.coef = -1.5 * c->cfg.omega_m / ((double)n * n * n);
    const int64_t rows = (int64_t)(n / 2 + 1) * n;
    auto run = [&](int form) -> cudaError_t {
        if (form == 0) {
            cudaError_t e = y_rows<float, false>(s0, rows, n, c->st);
            if (e == cudaSuccess) e = x_cols<float>(s0, s1, n / 2 + 1, n, op, c->st);
            if (e == cudaSuccess) e = y_rows_grad3<float>(s0, s1, s2, rows, n, c->kf, c->st);
            return e;
        }
        if (form == kFormPlane) return fft_plane<float>(s0, s1, s2, n / 2 + 1, n, op, c->st);
        return fft_middle<float>(s0, s1, s2, n / 2 + 1, n, op, (unsigned*)c->at(c->L.mid), form, c->st);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PM_CK(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    int best_t = 0;
    double best_ms = 1e30;
    for (size_t q = 0; q < cand.size() && err == cudaSuccess; ++q) {
        err = run(cand[q]);  // warm-up (and the one-time attribute set-up)
        for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
            err = cudaEventRecord(e0, c->st);
            if (err == cudaSuccess) err = run(cand[q]);
            if (err == cudaSuccess) err = cudaEventRecord(e1, c->st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                best_t = cand[q];
            }
        }
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return fail(PM_ERR_CUDA, std::string("pm_autotune_fft: ") + cudaGetErrorString(err));
    PM_TRY(check_wait_error(c));
    c->mid_threads = best_t;
    if (threads_out) *threads_out = best_t;
    if (ms_out) *ms_out = best_ms;
    return PM_OK;
}

pm_status pm_profile(pm_ctx* c, int enable) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    c->prof = enable != 0;
    return PM_OK;
}

pm_status pm_timings(pm_ctx* c, double* ms, int64_t* launches) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    PM_TRY(check_wait_error(c));
    double acc[PM_NPHASES] = {0};
    int64_t cnt[PM_NPHASES] = {0};
    for (auto& r : c->recs) {
        float t = 0.0f;
        PM_CK(cudaEventElapsedTime(&t, r.a, r.b));
        acc[r.phase] += t;
        cnt[r.phase] += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    for (int i = 0; i < PM_NPHASES; ++i) {
        if (ms) ms[i] = acc[i];
        if (launches) launches[i] = cnt[i];
    }
    return PM_OK;
}

pm_status pm_density(pm_ctx* c, void* delta) {
    if (!c || !delta) return fail(PM_ERR_INVALID_ARG, "null argument");
    const int64_t n3 = (int64_t)c->n * c->n * c->n;
    PM_CK(fill(delta, n3, c->cfg.precision, -1.0, c->st));
    PM_CK(deposit_lattice(c->at(c->L.x), c->np, c->cfg.precision, c->n, std::pow((double)c->n / c->np, 3), delta,
                          c->st));
    return PM_OK;
}

pm_status pm_potential(pm_ctx* c, void* phi) {
    if (!c || !phi) return fail(PM_ERR_INVALID_ARG, "null argument");
    const int n = c->n;
    const void* rho = nullptr;
    PM_TRY(current_density(c, &rho));
    SpecOp op;
    op.kind = OP_POTENTIAL;
    op.fwd = 1;
    op.kf = c->kf;
    op.coef = -1.5 * c->cfg.omega_m / ((double)n * n * n);
    if (c->fp64()) {
        double2* s0 = (double2*)c->at(c->L.spec[0]);
        PM_TRY(forward_to_y<double>(c, rho, s0, n, kDensityMean));
        PM_CK(x_cols<double>(s0, nullptr, n / 2 + 1, n, op, c->st));
        PM_CK((y_rows<double, true>(s0, (int64_t)(n / 2 + 1) * n, n, c->st)));
        const double2* in[1] = {s0};
        double* out[1] = {(double*)phi};
        PM_CK(z_c2r<double>(in, out, 1, n, 1, 0u, 0.0, c->st));
    } else {
        float2* s0 = (float2*)c->at(c->L.spec[0]);
        PM_TRY(forward_to_y<float>(c, rho, s0, n, kDensityMean));
        PM_CK(x_cols<float>(s0, nullptr, n / 2 + 1, n, op, c->st));
        PM_CK((y_rows<float, true>(s0, (int64_t)(n / 2 + 1) * n, n, c->st)));
        const float2* in[1] = {s0};
        float* out[1] = {(float*)phi};
        PM_CK(z_c2r<float>(in, out, 1, n, 1, 0u, 0.0, c->st));
    }
    return PM_OK;
}

pm_status pm_displacement_correction(pm_ctx* target, const pm_ctx* gr, const pm_ctx* newton, void* xi_out) {
    if (!target || !gr || !newton) return fail(PM_ERR_INVALID_ARG, "null context");
    if (gr->np != newton->np || gr->cfg.precision != newton->cfg.precision ||
        target->cfg.precision != gr->cfg.precision)
        return fail(PM_ERR_INVALID_ARG, "gr and newton must share np; all three must share precision");
    if (target->np < gr->np || target->np % gr->np)
        return fail(PM_ERR_INVALID_ARG, "target lattice must be a power-of-two multiple of the gr/newton lattice");
    if (gr->st != target->st) PM_CK(cudaStreamSynchronize(gr->st));
    if (newton->st != target->st) PM_CK(cudaStreamSynchronize(newton->st));
    PM_CK(combine(target->at(target->L.x), gr->at(gr->L.x), newton->at(newton->L.x), xi_out, target->np, gr->np,
                  target->cfg.precision, target->st));
    target->rho_valid = false;
    if (target->adj) target->adj->recorded = false;
    return PM_OK;
}

pm_status pm_power(pm_ctx* c, const void* field, const void* field2, int nbins, const double* edges, int deconvolve,
                   double* k_out, double* p_out, double* nmodes_out) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    PM_TRY(check_edges(nbins, edges));
    PM_TRY(check_wait_error(c));
    return c->fp64() ? power_t<double>(c, field, field2, nbins, edges, deconvolve, k_out, p_out, nmodes_out)
                     : power_t<float>(c, field, field2, nbins, edges, deconvolve, k_out, p_out, nmodes_out);
}

pm_status pm_halo_proxy(pm_ctx* c, const void* field, double fraction, void* delta_h, int64_t* selected) {
    if (!c || !delta_h) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (!(fraction > 0.0 && fraction <= 1.0)) return fail(PM_ERR_INVALID_ARG, "fraction must be in (0, 1]");
    const int64_t n3 = (int64_t)c->n * c->n * c->n;
    if (n3 > 0xFFFFFFFFll) return fail(PM_ERR_INVALID_ARG, "mesh too large for 32-bit ranks");
    const int64_t K = (int64_t)std::ceil(fraction * (double)n3);
    const void* f = field;
    if (!f) {
        c->rho_valid = false;  // rho is about to hold delta = rho - 1
        PM_CK(fill(c->at(c->L.rho), n3, c->cfg.precision, -1.0, c->st));
        PM_CK(deposit_lattice(c->at(c->L.x), c->np, c->cfg.precision, c->n, std::pow((double)c->n / c->np, 3),
                              c->at(c->L.rho), c->st));
        f = c->at(c->L.rho);
    }
    // spectrum buffers are free outside a step and serve as scratch
    if (halo_proxy_scratch_bytes(n3) > c->scratch_bytes)
        return fail(PM_ERR_WORKSPACE, "workspace too small for the selection");
    void* scratch = c->at(c->scratch_off);
    if (c->fp64())
        PM_CK(halo_proxy<double>((const double*)f, n3, K, (double*)delta_h, scratch, c->st));
    else
        PM_CK(halo_proxy<float>((const float*)f, n3, K, (float*)delta_h, scratch, c->st));
    if (selected) *selected = K;
    return PM_OK;
}

pm_status pm_linear_bias(pm_ctx* c, const void* delta_h, const void* delta_m, int nbins, const double* edges,
                         double k_max, int terms, double* coef, double* k_out, double* ratio_out, double* nmodes_out) {
    if (!c || !delta_h || !delta_m || !coef) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (terms < 1 || terms > 3) return fail(PM_ERR_INVALID_ARG, "terms must be 1 (b1), 2 (+ b1GR) or 3 (+ k^2)");
    PM_TRY(check_edges(nbins, edges));
    std::vector<double> k(nbins), phm(nbins), pmm(nbins), nm(nbins);
    // P_hm and P_mm from one pass over the two transforms
    PM_TRY(c->fp64() ? power_t<double>(c, delta_h, delta_m, nbins, edges, 1, k.data(), phm.data(), nm.data(), pmm.data())
                     : power_t<float>(c, delta_h, delta_m, nbins, edges, 1, k.data(), phm.data(), nm.data(), pmm.data()));
    const double a = c->a_grid(c->step);
    const double H = pmhost::conformal_hubble(c->cosmo, a);
    // weighted least squares (weights = mode counts) of P_hm/P_mm = b1 [+ b1GR H^2/k^2] [+ c k^2] on k < k_max
    double AtA[3][3] = {{0}}, Atb[3] = {0};
    int used = 0;
    for (int b = 0; b < nbins; ++b) {
        const double r = phm[b] / pmm[b];
        if (ratio_out) ratio_out[b] = r;
        if (k_out) k_out[b] = k[b];
        if (nmodes_out) nmodes_out[b] = nm[b];
        if (!(nm[b] > 0) || !std::isfinite(r) || !(k[b] < k_max)) continue;
        const double row[3] = {1.0, H * H / (k[b] * k[b]), k[b] * k[b]};
        for (int i = 0; i < terms; ++i) {
            Atb[i] += nm[b] * row[i] * r;
            for (int j = 0; j < terms; ++j) AtA[i][j] += nm[b] * row[i] * row[j];
        }
        ++used;
    }
    if (used < terms) return fail(PM_ERR_INVALID_ARG, "fewer usable bins than fit parameters");
    // Gaussian elimination with partial pivoting
    for (int i = 0; i < terms; ++i) {
        int piv = i;
        for (int r = i + 1; r < terms; ++r)
            if (std::fabs(AtA[r][i]) > std::fabs(AtA[piv][i])) piv = r;
        for (int j = 0; j < terms; ++j) std::swap(AtA[i][j], AtA[piv][j]);
        std::swap(Atb[i], Atb[piv]);
        if (AtA[i][i] == 0.0) return fail(PM_ERR_INVALID_ARG, "singular bias fit");
        for (int r = i + 1; r < terms; ++r) {
            const double fct = AtA[r][i] / AtA[i][i];
            for (int j = i; j < terms; ++j) AtA[r][j] -= fct * AtA[i][j];
            Atb[r] -= fct * Atb[i];
        }
    }
    for (int i = terms - 1; i >= 0; --i) {
        double s = Atb[i];
        for (int j = i + 1; j < terms; ++j) s -= AtA[i][j] * coef[j];
        coef[i] = s / AtA[i][i];
    }
    return PM_OK;
}

pm_status pm_bispectrum_scratch_size(const pm_ctx* c, int m, int nbins, size_t* bytes) {
    if (!c || !bytes) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (!pow2(m) || m < 16 || m > 1024) return fail(PM_ERR_INVALID_ARG, "m must be a power of two in 16..1024");
    if (nbins < 1 || nbins > 64) return fail(PM_ERR_INVALID_ARG, "bispectrum needs 1..64 bins");
    *bytes = bk_plan((int)c->sT(), m, nbins).total;
    return PM_OK;
}

pm_status pm_triangle_index(int nbins, int i, int j, int l, int64_t* index) {
    if (!index) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (nbins < 1 || i < 0 || i > j || j > l || l >= nbins) return fail(PM_ERR_INVALID_ARG, "not a triangle i <= j <= l");
    int64_t before = 0;
    for (int a = 0; a < i; ++a) before += (int64_t)(nbins - a) * (nbins - a + 1) / 2;  // (j, l) pairs with a <= j <= l
    for (int b = i; b < j; ++b) before += nbins - b;                                  // l in [b, nbins)
    *index = before + (l - j);
    return PM_OK;
}

pm_status pm_bispectrum(pm_ctx* c, const void* field, int nbins, const double* edges, int m, int deconvolve,
                        void* scratch, size_t scratch_bytes, double* b_out, double* ntri_out) {
    if (!c) return fail(PM_ERR_INVALID_ARG, "null context");
    PM_TRY(check_edges(nbins, edges));
    size_t need = 0;
    PM_TRY(pm_bispectrum_scratch_size(c, m, nbins, &need));
    if (!scratch || scratch_bytes < need || (uintptr_t)scratch % 256)
        return fail(PM_ERR_WORKSPACE, "bispectrum scratch too small or not 256-byte aligned");
    const int nmax = std::min((int)std::floor(edges[nbins]), c->n / 2 - 1);
    if (3 * nmax >= m) return fail(PM_ERR_INVALID_ARG, "grid m too small for an alias-free triangle sum");
    const BkLayout B = bk_plan((int)c->sT(), m, nbins);
    return c->fp64() ? bispectrum_t<double>(c, field, nbins, edges, m, deconvolve, (unsigned char*)scratch, B, b_out,
                                            ntri_out)
                     : bispectrum_t<float>(c, field, nbins, edges, m, deconvolve, (unsigned char*)scratch, B, b_out,
                                           ntri_out);
}

}  // extern "C"


// ====================================================================== gradient of a field loss
namespace {

struct AdjLayout {
    // two segment records (positions and force meshes of C steps) so that the re-run of one
    // segment overlaps the reverse sweep of the next; the re-runs' own density, spectra and
    // end positions
    size_t ckpt = 0, seg_x[2] = {0, 0}, seg_g[2] = {0, 0}, lam_u = 0, lam_p = 0, acc = 0;
    size_t re_rho = 0, re_spec[3] = {0, 0, 0}, re_x = 0, close_g = 0, total = 0;
    // Poisson gauge: Phi_old and the FP64 island at every checkpoint, the re-runs' own, and
    // the carried spectrum Z of the transposed lagged constraint
    size_t ckpt_phi = 0, ckpt_isl = 0, re_phi = 0, re_isl = 0, zcarry = 0, isl = 0;
    int nseg = 0, C = 0;
};

AdjLayout adj_plan(const pm_ctx* c, int C) {
    AdjLayout A;
    const int S = c->cfg.n_steps;
    A.C = C;
    A.nseg = (S + C - 1) / C;
    const size_t P = 3 * (size_t)c->np3 * 4, G = 3 * (size_t)c->n * c->n * c->n * 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t n = c->n, spec = 2 * (n / 2 + 1) * n * n * 4;
    A.ckpt = take((size_t)A.nseg * 2 * P);
    for (int b = 0; b < 2; ++b) {
        A.seg_x[b] = take((size_t)C * P);
        A.seg_g[b] = take((size_t)C * G);
    }
    A.lam_u = take(P);
    A.lam_p = take(P);
    A.acc = take(8);
    A.re_rho = take(n * n * n * 4);
    for (int j = 0; j < 3; ++j) A.re_spec[j] = take(spec);
    A.re_x = take(P);
    A.close_g = take(G);  // the force meshes of the closing half kick
    if (c->L.gr) {
        A.isl = c->L.has_island ? (size_t)(c->cfg.n_lo + 1) * (2 * c->cfg.n_lo + 1) * (2 * c->cfg.n_lo + 1) * 16 : 0;
        A.ckpt_phi = take((size_t)A.nseg * spec);
        A.ckpt_isl = take((size_t)A.nseg * A.isl);
        A.re_phi = take(spec);
        A.re_isl = take(A.isl);
        A.zcarry = take(spec);
    }
    A.total = off;
    return A;
}

// Forward transforms of `batch` real meshes of side n stored back to back into as many
// spectra ([kz][kx][ky]) stored back to back.
pm_status fft_forward_f32(pm_ctx* c, const float* real, float2* spec, int n, int batch = 1) {
    PM_CK(z_r2c<float>(real, spec, n, batch, c->st));
    PM_CK((y_rows<float, false>(spec, (int64_t)batch * (n / 2 + 1) * n, n, c->st)));
    SpecOp fw;
    fw.kind = OP_FWD_STORE;
    fw.fwd = 1;
    PM_CK(x_cols<float>(spec, nullptr, batch * (n / 2 + 1), n, fw, c->st));
    return PM_OK;
}

pm_status fft_inverse_f32(pm_ctx* c, float2* spec, float* real, int n) {
    SpecOp inv;
    inv.kind = OP_INV;
    inv.fwd = 0;
    PM_CK(x_cols<float>(spec, nullptr, n / 2 + 1, n, inv, c->st));
    PM_CK((y_rows<float, true>(spec, (int64_t)(n / 2 + 1) * n, n, c->st)));
    const float2* in[1] = {spec};
    float* out[1] = {real};
    PM_CK(z_c2r<float>(in, out, 1, n, 1, 0u, 0.0, c->st));
    return PM_OK;
}

// lambda_u += K J(u)^T lambda_p at positions xs with force meshes gs (three n^3 meshes),
// then lambda_p += drift_next lambda_u (the transposed drift of the step before; 0: none).
// V (the context's force meshes) is zero on entry and left zero.
pm_status adj_kick(pm_ctx* c, const uint32_t* xs, const float* gs, double K, float* lam_u, float* lam_p,
                   double drift_next, const AdjGrOp* gr = nullptr) {
    const int n = c->n;
    const size_t n3 = (size_t)n * n * n;
    const float* G[3] = {gs, gs + n3, gs + 2 * n3};
    // V_j and the spectra are three meshes back to back (256-byte multiples): one batched transform
    float* V[3] = {(float*)c->at(c->L.force[0]), (float*)c->at(c->L.force[1]), (float*)c->at(c->L.force[2])};
    const double mass = std::pow((double)n / c->np, 3);
    if (c->cfg.gradient == PM_GRAD_FD1) {
        // first-order gradient: gs[0] is the recorded potential; one scalar deposit with the CIC
        // derivative weights, its transposed potential map, then the particle side
        const double inv_d = n / c->cfg.box;
        float2* s0 = (float2*)c->at(c->L.spec[0]);
        PM_CK(deposit_grad(xs, c->np3, n, lam_p, inv_d, V[0], c->st));
        PM_CK(forward_zy<float>(V[0], s0, n, 1, c->st));
        PM_CK(x_adj<float>(s0, s0, n, c->kf, -1.5 * c->cfg.omega_m / ((double)n * n * n), c->st, V[0], (int64_t)n3, gr,
                           true));
        float* rho_bar = (float*)c->at(c->L.rho);
        PM_CK((y_rows<float, true>(s0, (int64_t)(n / 2 + 1) * n, n, c->st)));
        const float2* zin[1] = {s0};
        float* zout[1] = {rho_bar};
        PM_CK(z_c2r<float>(zin, zout, 1, n, 1, 0u, 0.0, c->st));
        PM_CK(adj_kick_particles_fd(xs, c->np3, n, lam_p, gs, rho_bar, (float)K, (float)(gr ? mass : K * mass), inv_d,
                                    (float)drift_next, lam_u, c->st));
        return PM_OK;
    }
    PM_CK(deposit_vec(xs, c->np, n, lam_p, V, c->st));
    float2* sp[3] = {(float2*)c->at(c->L.spec[0]), (float2*)c->at(c->L.spec[1]), (float2*)c->at(c->L.spec[2])};
    // forward z and y passes of the three meshes, then the x pass that combines them
    // (sum_j i k_j C V_j), transforms back and clears V for the next deposit, then the
    // inverse y and z passes
    PM_CK(forward_zy<float>(V[0], sp[0], n, 3, c->st));
    // in place over field 0: each CTA reads and writes only its own columns
    PM_CK(x_adj<float>(sp[0], sp[0], n, c->kf, -1.5 * c->cfg.omega_m / ((double)n * n * n), c->st, V[0],
                       3 * (int64_t)n3, gr));
    float* rho_bar = (float*)c->at(c->L.rho);
    PM_CK((y_rows<float, true>(sp[0], (int64_t)(n / 2 + 1) * n, n, c->st)));
    const float2* zin[1] = {sp[0]};
    float* zout[1] = {rho_bar};
    PM_CK(z_c2r<float>(zin, zout, 1, n, 1, 0u, 0.0, c->st));
    // Newtonian: rho_bar lacks this evaluation's K; Poisson gauge: Z carries every K already
    PM_CK(adj_kick_particles(xs, c->np3, n, lam_p, G, rho_bar, (float)K, (float)(gr ? mass : K * mass),
                             (float)drift_next, lam_u, c->st));
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_adjoint_scratch_size(const pm_ctx* c, int checkpoint_every, size_t* bytes) {
    if (!c || !bytes || checkpoint_every < 1) return fail(PM_ERR_INVALID_ARG, "bad arguments");
    *bytes = adj_plan(c, std::min(checkpoint_every, c->cfg.n_steps)).total;
    return PM_OK;
}

}  // extern "C"

namespace {

double kick_of_step(const pm_ctx* c, int s) {
    const double a0 = c->a_grid(s), a1 = c->a_grid(s + 1);
    const double a_from = (s == 0) ? a0 : 0.5 * (c->a_grid(s - 1) + a0);
    return kick_factor(c->cfg, c->cosmo, a_from, 0.5 * (a0 + a1), a0);
}
double drift_of_step(const pm_ctx* c, int s) {
    const double a0 = c->a_grid(s), a1 = c->a_grid(s + 1);
    return drift_factor(c->cfg, c->cosmo, a0, a1, 0.5 * (a0 + a1));
}

// Pieces of the reverse sweep shared by pm_adjoint_record, pm_adjoint_run and pm_loss_grad.
// Layout A of the scratch; record k & 1 holds the positions and force meshes of segment k.
struct AdjSweep {
    pm_ctx* c;
    pm_ctx::AdjSession& S;
    AdjLayout A;
    int steps;
    size_t P, Gb;
    AdjSweep(pm_ctx* ctx, pm_ctx::AdjSession& s) : c(ctx), S(s) {
        steps = c->cfg.n_steps;
        A = adj_plan(c, S.C);
        P = 3 * (size_t)c->np3 * 4;
        Gb = 3 * (size_t)c->n * c->n * c->n * 4;
    }
    void* at(size_t off) const { return (unsigned char*)S.scratch + off; }
    void* seg_x(int k, int i) const { return at(A.seg_x[k & 1] + (size_t)i * P); }
    void* seg_g(int k, int i) const { return at(A.seg_g[k & 1] + (size_t)i * Gb); }
    void* ckpt_x(int k) const { return at(A.ckpt + (size_t)k * 2 * P); }
    void* ckpt_p(int k) const { return at(A.ckpt + (size_t)k * 2 * P + P); }
    size_t spec_bytes() const { return 2 * (size_t)(c->n / 2 + 1) * c->n * c->n * 4; }
    void* ckpt_phi(int k) const { return at(A.ckpt_phi + (size_t)k * spec_bytes()); }
    void* ckpt_isl(int k) const { return at(A.ckpt_isl + (size_t)k * A.isl); }

    // Poisson gauge: the transposed operator of force evaluation e (steps e = 0 .. steps - 1
    // at a_e, the closing kick e = steps at a_final) with kick factor K; its scalars as the
    // forward evaluation forms them (dtau from the previous evaluation), and those of e + 1.
    AdjGrOp gr_op(int e, double K) const {
        AdjGrOp g;
        auto scalars = [&](int i, double& H, double& om, double& cc) {
            const double a = c->a_grid(i);
            H = pmhost::conformal_hubble(c->cosmo, a);
            om = pmhost::omega_m_a(c->cosmo, a);
            cc = i > 0 ? 3.0 * H / (pmhost::kCLight * pmhost::kick_integral(c->cosmo, c->a_grid(i - 1), a)) : 0.0;
        };
        scalars(e, g.H, g.om, g.cc);
        if (e < steps) scalars(e + 1, g.H1, g.om1, g.cc1);
        else g.H1 = g.H, g.om1 = g.om, g.cc1 = 0.0;  // nothing after the closing kick: Z is 0 there
        const double n3 = (double)c->n * c->n * c->n;
        g.K_ac2_n3 = K * c->a_grid(e) * pmhost::kCLight * pmhost::kCLight / n3;
        g.Z = at(A.zcarry);
        return g;
    }

    // Steps s0..s1-1 of segment k on context r from the positions at rx (p in place), keeping
    // each step's positions and force meshes in record k & 1.  With the fused update each
    // step reads its positions from the record and writes the drifted ones into the next
    // slot (the last step's to x_end), so only the segment's first positions are copied.
    pm_status record(pm_ctx* r, int k, void* rx, void* x_end) const {
        const int s0 = k * S.C, s1 = std::min(steps, s0 + S.C);
        const bool oop = fused_update(c);
        if (oop) PM_CK(cudaMemcpyAsync(seg_x(k, 0), rx, P, cudaMemcpyDeviceToDevice, r->st));
        for (int s = s0; s < s1; ++s) {
            void* xs = seg_x(k, s - s0);
            if (oop) {
                r->x_at = xs;
                r->x_out = (s + 1 < s1) ? seg_x(k, s + 1 - s0) : x_end;
            } else {
                PM_CK(cudaMemcpyAsync(xs, r->xpos(), P, cudaMemcpyDeviceToDevice, r->st));
            }
            r->force_at = seg_g(k, s - s0);
            pm_status st = compute_forces(r, r->a_grid(s));
            if (st == PM_OK) st = kick_drift(r, kick_of_step(r, s), drift_of_step(r, s));
            r->force_at = nullptr;
            r->x_at = r->x_out = nullptr;
            if (st != PM_OK) return st;
            r->step = s + 1;
            r->synced = false;
        }
        return PM_OK;
    }

    // The forward run from the ICs of white noise w with checkpoints of (x, p) before every
    // segment; the last two segments are recorded as they run (one record each), so the
    // reverse sweep starts without a re-run.  Then the closing half kick synchronises the
    // momenta, as at the end of any run, with its force meshes kept for the reverse sweep of
    // a momentum cotangent.
    pm_status forward(const void* white_noise) const {
        PM_TRY(pm_ic_zeldovich(c, 0, white_noise, 0));
        void* x = c->at(c->L.x);
        void* p = c->at(c->L.p);
        for (int k = 0; k < A.nseg; ++k) {
            const int s0 = k * S.C, s1 = std::min(steps, s0 + S.C);
            PM_CK(cudaMemcpyAsync(ckpt_x(k), x, P, cudaMemcpyDeviceToDevice, c->st));
            PM_CK(cudaMemcpyAsync(ckpt_p(k), p, P, cudaMemcpyDeviceToDevice, c->st));
            if (c->L.gr && k > 0) {  // the lagged constraint's history at the segment's start
                PM_CK(cudaMemcpyAsync(ckpt_phi(k), c->at(c->L.phi_old), spec_bytes(), cudaMemcpyDeviceToDevice,
                                      c->st));
                if (A.isl)
                    PM_CK(cudaMemcpyAsync(ckpt_isl(k), c->at(c->L.island), A.isl, cudaMemcpyDeviceToDevice, c->st));
            }
            PM_CK(cudaEventRecord(S.ev_ckpt[k], c->st));
            if (k < A.nseg - 2) PM_TRY(pm_step(c, s1 - s0));
            else PM_TRY(record(c, k, x, x));
        }
        c->force_at = at(A.close_g);
        pm_status st = compute_forces(c, c->a_grid(steps));
        if (st == PM_OK) st = kick_drift(c, close_kick(), 0.0);
        c->force_at = nullptr;
        PM_TRY(st);
        c->synced = true;
        c->rho_valid = false;
        return PM_OK;
    }
    double close_kick() const {
        return kick_factor(c->cfg, c->cosmo, 0.5 * (c->a_grid(steps - 1) + c->a_grid(steps)), c->a_grid(steps),
                           c->a_grid(steps));
    }

    // Reverse sweep from the adjoint positions lam_u (scratch lam_u) and, with mom, the adjoint
    // momenta in scratch lam_p (else lam_p = 0 after the closing kick) down to dL/dw.  Every segment before the last two is re-run from its
    // checkpoint on the second stream, on a context of its own (density and spectra in the
    // scratch, p and, without the fused update, x in place over the checkpoint, which is
    // used once), into the record the reverse sweep of the segment after it has just
    // released; events order the two streams.
    pm_status reverse(void* grad_out, bool mom) const {
        const double box = c->cfg.box;
        float* lam_u = (float*)at(A.lam_u);
        float* lam_p = (float*)at(A.lam_p);
        pm_ctx re = *c;
        re.pool.clear();
        re.recs.clear();
        re.prof = false;
        re.st = c->st2;
        re.st2 = nullptr;
        re.adj = nullptr;
        // its workspace is the scratch: no sync words of its own there for the persistent form
        re.mid_threads = (c->mid_threads == kFormPlane) ? kFormPlane : 0;
        re.ws = (unsigned char*)S.scratch;
        re.L.rho = A.re_rho;
        for (int j = 0; j < 3; ++j) re.L.spec[j] = A.re_spec[j];
        re.L.phi_old = A.re_phi;
        re.L.island = A.re_isl;
        auto rerun = [&](int k) -> pm_status {
            PM_CK(cudaStreamWaitEvent(re.st, S.ev_ckpt[k], 0));
            if (k + 2 < A.nseg) PM_CK(cudaStreamWaitEvent(re.st, S.ev_rev[k + 2], 0));  // record k & 1 is free
            re.L.x = A.ckpt + (size_t)k * 2 * P;
            re.L.p = re.L.x + P;
            re.step = k * S.C;
            re.synced = (k == 0);
            re.rho_valid = false;
            if (c->L.gr) {  // the lagged constraint resumes from the checkpoint's history
                re.have_phi = k > 0;
                re.a_last = k > 0 ? c->a_grid(k * S.C - 1) : 0.0;
                if (k > 0) {
                    PM_CK(cudaMemcpyAsync(re.at(re.L.phi_old), ckpt_phi(k), spec_bytes(), cudaMemcpyDeviceToDevice,
                                          re.st));
                    if (A.isl)
                        PM_CK(cudaMemcpyAsync(re.at(re.L.island), ckpt_isl(k), A.isl, cudaMemcpyDeviceToDevice,
                                              re.st));
                }
            }
            PM_TRY(record(&re, k, re.at(re.L.x), at(A.re_x)));
            PM_CK(cudaEventRecord(S.ev_rerun[k], re.st));
            return PM_OK;
        };
        // V (the three force meshes, back to back) is zero before the first adjoint deposit,
        // and so is the carried spectrum of the Poisson gauge before the last evaluation
        PM_CK(cudaMemsetAsync(c->at(c->L.force[0]), 0, Gb, c->st));
        const bool gr = c->L.gr;
        if (gr) PM_CK(cudaMemsetAsync(at(A.zcarry), 0, spec_bytes(), c->st));
        // the transposed closing kick at the final positions (only a momentum cotangent sees
        // it), then the transposed drift of the last step gives lam_p
        if (mom) {
            const AdjGrOp og = gr_op(steps, close_kick());
            PM_TRY(adj_kick(c, (const uint32_t*)c->at(c->L.x), (const float*)at(A.close_g), close_kick(), lam_u, lam_p,
                            drift_of_step(c, steps - 1) / box, gr ? &og : nullptr));
        } else {
            PM_CK(axpby(lam_p, lam_u, nullptr, 3 * c->np3, (float)(drift_of_step(c, steps - 1) / box), 0.0f, c->st));
        }
        for (int k = A.nseg - 1; k >= 0; --k) {
            const int s0 = k * S.C, s1 = std::min(steps, s0 + S.C);
            if (k < A.nseg - 2) PM_CK(cudaStreamWaitEvent(c->st, S.ev_rerun[k], 0));
            for (int s = s1 - 1; s >= s0; --s) {
                const AdjGrOp og = gr_op(s, kick_of_step(c, s));
                PM_TRY(adj_kick(c, (const uint32_t*)seg_x(k, s - s0), (const float*)seg_g(k, s - s0),
                                kick_of_step(c, s), lam_u, lam_p, s > 0 ? drift_of_step(c, s - 1) / box : 0.0,
                                gr ? &og : nullptr));
            }
            PM_CK(cudaEventRecord(S.ev_rev[k], c->st));
            if (k >= 2) PM_TRY(rerun(k - 2));
        }
        // transposed Zel'dovich map: grad = sum_j A_j^T (D/L lam_u_j + a^2 E f D lam_p_j)
        const int np = c->np;
        const double a = c->cfg.a_init;
        const double D = pmhost::growth_D(c->cosmo, a), f = pmhost::growth_f(c->cosmo, a), E = pmhost::E(c->cosmo, a);
        const int64_t np3 = c->np3;
        float* s_j[3] = {(float*)c->at(c->L.force[0]), (float*)c->at(c->L.force[1]), (float*)c->at(c->L.force[2])};
        float2* sp[3] = {(float2*)c->at(c->L.spec[0]), (float2*)c->at(c->L.spec[1]), (float2*)c->at(c->L.spec[2])};
        for (int j = 0; j < 3; ++j) {
            PM_CK(axpby(s_j[j], lam_u + j * np3, lam_p + j * np3, np3, (float)(D / box), (float)(a * a * E * f * D),
                        c->st));
            PM_TRY(fft_forward_f32(c, s_j[j], sp[j], np));
        }
        const float2* in[3] = {sp[0], sp[1], sp[2]};
        PM_CK(adj_combine(in, sp[0], np, c->kf, -std::pow((double)np, -1.5), (const double*)c->at(c->L.amp), 1,
                          c->st));
        PM_TRY(fft_inverse_f32(c, sp[0], (float*)grad_out, np));
        return PM_OK;
    }
};

// Checks shared by the entry points of the reverse sweep; creates the second stream and
// the session's events for checkpoint interval C.
pm_status adj_prepare(pm_ctx* c, int checkpoint_every, void* scratch, size_t scratch_bytes) {
    if (checkpoint_every < 1) return fail(PM_ERR_INVALID_ARG, "bad checkpoint interval");
    if (c->cfg.precision != PM_FP32_FIXED)
        return fail(PM_ERR_UNSUPPORTED, "the gradient is implemented for the FP32 step");
    const int C = std::min(checkpoint_every, c->cfg.n_steps);
    const AdjLayout A = adj_plan(c, C);
    if (!scratch || scratch_bytes < A.total || (uintptr_t)scratch % 256)
        return fail(PM_ERR_WORKSPACE, "adjoint scratch too small or not 256-byte aligned");
    if (!c->st2) PM_CK(cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking));
    if (!c->adj) c->adj = new pm_ctx::AdjSession();
    pm_ctx::AdjSession& S = *c->adj;
    S.scratch = scratch;
    S.bytes = scratch_bytes;
    S.C = C;
    S.recorded = false;
    for (auto* v : {&S.ev_ckpt, &S.ev_rerun, &S.ev_rev}) {
        while ((int)v->size() < A.nseg) {
            cudaEvent_t e = nullptr;
            PM_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            v->push_back(e);
        }
    }
    return PM_OK;
}

// After an error the second stream may still run a re-run into the scratch: wait for it
// before the scratch goes back to the caller.
void adj_settle(pm_ctx* c) {
    if (c->st2) cudaStreamSynchronize(c->st2);
}

}  // namespace

extern "C" {

pm_status pm_adjoint_record(pm_ctx* c, const void* white_noise, int checkpoint_every, void* scratch,
                            size_t scratch_bytes) {
    if (!c || !white_noise) return fail(PM_ERR_INVALID_ARG, "null argument");
    PM_TRY(adj_prepare(c, checkpoint_every, scratch, scratch_bytes));
    AdjSweep sw(c, *c->adj);
    pm_status st = sw.forward(white_noise);
    if (st != PM_OK) {
        adj_settle(c);
        return st;
    }
    c->adj->recorded = true;
    return PM_OK;
}

pm_status pm_adjoint_run(pm_ctx* c, const void* d_delta, const void* d_disp, const void* d_mom, void* grad_w) {
    if (!c || !grad_w || (!d_delta && !d_disp && !d_mom)) return fail(PM_ERR_INVALID_ARG, "null argument");
    if (!c->adj || !c->adj->recorded || c->step != c->cfg.n_steps)
        return fail(PM_ERR_STATE, "pm_adjoint_run needs the forward run of pm_adjoint_record first");
    pm_ctx::AdjSession& S = *c->adj;
    S.recorded = false;  // the re-runs overwrite the checkpoints: one reverse sweep per record
    AdjSweep sw(c, S);
    const int64_t m = 3 * c->np3;
    float* lam_u = (float*)sw.at(sw.A.lam_u);
    float* tmp = (float*)sw.at(sw.A.lam_p);
    const double mass = std::pow((double)c->n / c->np, 3);
    auto body = [&]() -> pm_status {
        // lam_u = m sum_c dL/ddelta(c) dW(x, c)/du + L dL/d(disp), u in box units
        if (d_delta) {
            PM_CK(adj_gather((const uint32_t*)c->at(c->L.x), c->np3, c->n, (const float*)d_delta, (float)mass, 0,
                             lam_u, c->st));
            if (d_disp) {
                PM_CK(axpby(tmp, lam_u, (const float*)d_disp, m, 1.0f, (float)c->cfg.box, c->st));
                PM_CK(axpby(lam_u, tmp, nullptr, m, 1.0f, 0.0f, c->st));
            }
        } else if (d_disp) {
            PM_CK(axpby(lam_u, (const float*)d_disp, nullptr, m, (float)c->cfg.box, 0.0f, c->st));
        } else {
            PM_CK(cudaMemsetAsync(lam_u, 0, sizeof(float) * m, c->st));
        }
        // lam_p = dL/dp of the synchronised final momenta (tmp was scratch until here)
        if (d_mom) PM_CK(axpby(tmp, (const float*)d_mom, nullptr, m, 1.0f, 0.0f, c->st));
        return sw.reverse(grad_w, d_mom != nullptr);
    };
    pm_status st = body();
    if (st == PM_OK) {
        cudaError_t e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) st = fail(PM_ERR_CUDA, cudaGetErrorString(e));
    }
    adj_settle(c);
    c->rho_valid = false;
    return st;
}

pm_status pm_loss_grad(pm_ctx* c, const void* white_noise, const void* target, int checkpoint_every, void* scratch,
                       size_t scratch_bytes, double* loss_out, void* grad_out) {
    if (!c || !white_noise || !target || !loss_out || !grad_out)
        return fail(PM_ERR_INVALID_ARG, "null argument or bad checkpoint interval");
    PM_TRY(pm_adjoint_record(c, white_noise, checkpoint_every, scratch, scratch_bytes));
    AdjSweep sw(c, *c->adj);
    const int64_t n3 = (int64_t)c->n * c->n * c->n;
    // the loss and its mesh adjoint 2 (delta - delta_t) / n^3, written over delta
    float* rho = (float*)c->at(c->L.rho);
    double* acc = (double*)sw.at(sw.A.acc);
    auto seed = [&]() -> pm_status {
        PM_CK(fill(rho, n3, PM_FP32_FIXED, -1.0, c->st));
        PM_CK(deposit_lattice(c->at(c->L.x), c->np, PM_FP32_FIXED, c->n, std::pow((double)c->n / c->np, 3), rho,
                              c->st));
        PM_CK(cudaMemsetAsync(acc, 0, 8, c->st));
        PM_CK(loss_mse(rho, (const float*)target, n3, acc, c->st));
        return PM_OK;
    };
    pm_status st = seed();
    if (st != PM_OK) {
        adj_settle(c);
        return st;
    }
    PM_TRY(pm_adjoint_run(c, rho, nullptr, nullptr, grad_out));
    double hsum = 0.0;
    PM_CK(cudaMemcpyAsync(&hsum, acc, 8, cudaMemcpyDeviceToHost, c->st));
    PM_CK(cudaStreamSynchronize(c->st));
    *loss_out = hsum / (double)n3;
    return PM_OK;
}

}  // extern "C"

// ====================================================================== batch of realisations
struct pm_batch {
    pm_config cfg;
    int B = 0;
    unsigned char* ws = nullptr;
    cudaStream_t st = nullptr;   // caller stream
    cudaStream_t cap = nullptr;  // library stream on which runs are captured into a graph
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_from = -1, exec_steps = 0;
    std::vector<pm_ctx*> views;  // one context per realisation on slices of the workspace
    size_t X = 0, P = 0, RHO = 0, SPEC[3] = {0, 0, 0}, FORCE[3] = {0, 0, 0}, AMP = 0, KF = 0, SCALE = 0;
    size_t BIN = 0, WTAB = 0, ACC = 0, total = 0;
    size_t PHI = 0, ISL = 0, isl = 0;  // Poisson gauge: Phi_old and the FP64 island of every realisation
    int64_t amp_len = 0;
    int step = 0;
    bool synced = true;
    bool rho_valid = false;
    int chunk = 0;  // realisations per launch of every pass (0: the whole batch)
    int fft_form = 0;  // middle FFT passes: 0 separate launches, 1 whole kz planes in shared memory
    bool have_ic = false;  // pm_batch_ic has run (the autotuner would overwrite the particles)
    pmhost::Cosmo cosmo;
    void* at(size_t off) const { return ws + off; }
    double a_grid(int i) const { return cfg.a_init + ((cfg.a_final - cfg.a_init) * i) / cfg.n_steps; }
    ~pm_batch() {
        for (auto* v : views) delete v;
        if (exec) cudaGraphExecDestroy(exec);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

void batch_plan(pm_batch& b) {
    const pm_config& c = b.cfg;
    const size_t np3 = (size_t)c.np * c.np * c.np, n = c.nmesh, n3 = n * n * n, nspec = (n / 2 + 1) * n * n;
    const size_t B = b.B;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    b.X = take(B * 3 * np3 * 4);
    b.P = take(B * 3 * np3 * 4);
    b.RHO = take(B * n3 * 4);
    for (int j = 0; j < 3; ++j) b.SPEC[j] = take(B * nspec * 8);
    for (int j = 0; j < 3; ++j) b.FORCE[j] = take(B * n3 * 4);
    b.amp_len = 3 * (int64_t)(c.np / 2) * (c.np / 2) + 1;
    b.AMP = take(B * b.amp_len * 8);
    b.KF = take(B * 8);
    b.SCALE = take(B * 8);
    b.BIN = take((3 * (n / 2) * (n / 2) + 1) * 2);
    b.WTAB = take((n / 2 + 1) * 8);
    b.ACC = take(2 * kMaxBins * 8);
    if (c.mode == PM_GR_POISSON) {
        b.PHI = take(B * nspec * 8);
        b.isl = c.n_lo > 0 ? (size_t)(c.n_lo + 1) * (2 * c.n_lo + 1) * (2 * c.n_lo + 1) * 16 : 0;
        b.ISL = take(B * b.isl);
    }
    b.total = off;
}

pm_status batch_validate(const pm_config* cfg, int B, const double* boxes) {
    PM_TRY(validate(cfg));
    if (B < 1 || B > 4096) return fail(PM_ERR_INVALID_ARG, "batch size must be in 1..4096");
    if (cfg->precision != PM_FP32_FIXED || cfg->gradient != PM_GRAD_SPECTRAL)
        return fail(PM_ERR_INVALID_ARG, "batches run the FP32 step with the spectral force");
    if (!ikd_deposit_supported(cfg->np, cfg->precision, cfg->nmesh))
        return fail(PM_ERR_INVALID_ARG, "batches need nmesh >= 64 and nmesh / np in {1, 2, 4}");
    if (boxes)
        for (int r = 0; r < B; ++r)
            if (!(boxes[r] > 0)) return fail(PM_ERR_INVALID_ARG, "box sizes must be positive");
    return PM_OK;
}

// Force meshes of realisations r0 .. r0 + c - 1 from their rho (one launch per pass).
pm_status batch_forces(pm_batch* b, cudaStream_t s, int r0, int c) {
    const int n = b->cfg.nmesh, M = n / 2;
    const size_t n3 = (size_t)n * n * n, nspec = (size_t)(M + 1) * n * n;
    float* rho = (float*)b->at(b->RHO) + r0 * n3;
    float2* s0 = (float2*)b->at(b->SPEC[0]) + r0 * nspec;
    float2* s1 = (float2*)b->at(b->SPEC[1]) + r0 * nspec;
    float2* s2 = (float2*)b->at(b->SPEC[2]) + r0 * nspec;
    const double* kf = (const double*)b->at(b->KF) + r0;
    const bool plane = b->fft_form == 1 && (n == 64 || n == 128);
    // rho, consumed by the forward z pass, receives the update's deposit next: the inverse z pass
    // clears it beside its force rows
    if (plane) PM_CK(z_r2c<float>(rho, s0, n, c, s, kDensityMean));
    else PM_CK(forward_zy<float>(rho, s0, n, c, s, kDensityMean));
    SpecOp op;
    op.kind = OP_NEWTON;
    op.fwd = 1;
    op.coef = -1.5 * b->cfg.omega_m / ((double)n * n * n);
    op.kf_arr = kf;
    if (b->cfg.mode == PM_GR_POISSON) {
        // force evaluation e = b->step (the closing kick's is n_steps) at a_e; its lagged
        // constraint reads the previous evaluation's Phi (a_{e-1}), none at the first
        const int e = b->step;
        const double a = b->a_grid(e);
        op.kind = OP_GR;
        op.calH = pmhost::conformal_hubble(b->cosmo, a);
        op.omm_a = pmhost::omega_m_a(b->cosmo, a);
        op.first = e == 0 ? 1 : 0;
        op.inv_dtau = e > 0 ? 1.0 / (pmhost::kCLight * pmhost::kick_integral(b->cosmo, b->a_grid(e - 1), a)) : 0.0;
        op.ac2_over_n3 = a * pmhost::kCLight * pmhost::kCLight / ((double)n * n * n);
        op.n_lo = b->cfg.n_lo;
        op.phi_old = (float2*)b->at(b->PHI) + r0 * nspec;
        op.island = b->isl ? (double2*)((unsigned char*)b->at(b->ISL) + r0 * b->isl) : nullptr;
    }
    float* out[3] = {(float*)b->at(b->FORCE[0]) + r0 * n3, (float*)b->at(b->FORCE[1]) + r0 * n3,
                     (float*)b->at(b->FORCE[2]) + r0 * n3};
    if (plane) {
        // whole kz planes in shared memory: the three gradient spectra, then the z pass
        PM_CK(fft_plane<float>(s0, s1, s2, c * (M + 1), n, op, s));
        const float2* in[3] = {s1, s2, s0};
        PM_CK(z_c2r<float>(in, out, 3, n, c, 0u, 0.0, s, nullptr, rho));
        return PM_OK;
    }
    PM_CK(x_cols<float>(s0, s1, c * (M + 1), n, op, s));
    PM_CK(inverse_yz_grad<float>(s0, s1, s2, out, n, c, 0.0, s, kf, rho));
    return PM_OK;
}

pm_status batch_update(pm_batch* b, double kick, double drift, cudaStream_t s, int r0, int c) {
    const size_t n3 = (size_t)b->cfg.nmesh * b->cfg.nmesh * b->cfg.nmesh;
    const size_t np3 = (size_t)b->cfg.np * b->cfg.np * b->cfg.np;
    void* g[3] = {(float*)b->at(b->FORCE[0]) + r0 * n3, (float*)b->at(b->FORCE[1]) + r0 * n3,
                  (float*)b->at(b->FORCE[2]) + r0 * n3};
    const double mass = std::pow((double)b->cfg.nmesh / b->cfg.np, 3);
    PM_CK(interp_kick_drift_deposit((uint32_t*)b->at(b->X) + r0 * 3 * np3, (float*)b->at(b->P) + r0 * 3 * np3,
                                    b->cfg.np, PM_FP32_FIXED, b->cfg.nmesh, g, kick, drift, 1.0, mass,
                                    (float*)b->at(b->RHO) + r0 * n3, s, c, (const double*)b->at(b->SCALE) + r0));
    return PM_OK;
}

// Forces and update of every realisation, chunk by chunk: each chunk's passes follow one
// another, so a chunk small enough for L2 keeps its meshes there between the passes.
pm_status batch_forces_update(pm_batch* b, double kick, double drift, cudaStream_t s) {
    const int c = (b->chunk > 0 && b->chunk < b->B) ? b->chunk : b->B;
    for (int r0 = 0; r0 < b->B; r0 += c) {
        const int cc = std::min(c, b->B - r0);
        PM_TRY(batch_forces(b, s, r0, cc));
        PM_TRY(batch_update(b, kick, drift, s, r0, cc));
    }
    return PM_OK;
}

// One KDK step of every realisation (the same a-grid for all), enqueued on s.
pm_status batch_enqueue_step(pm_batch* b, cudaStream_t s) {
    const double a0 = b->a_grid(b->step), a1 = b->a_grid(b->step + 1), ah = 0.5 * (a0 + a1);
    const double a_from = b->synced ? a0 : 0.5 * (b->a_grid(b->step - 1) + a0);
    PM_TRY(batch_forces_update(b, kick_factor(b->cfg, b->cosmo, a_from, ah, a0),
                               drift_factor(b->cfg, b->cosmo, a0, a1, ah), s));
    b->step += 1;
    b->synced = false;
    if (b->step == b->cfg.n_steps) {
        PM_TRY(batch_forces_update(b, kick_factor(b->cfg, b->cosmo, ah, a1, a1), 0.0, s));
        b->synced = true;
    }
    return PM_OK;
}

void batch_drop_graph(pm_batch* b) {
    if (b->exec) {
        cudaStreamSynchronize(b->cap);
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->exec_from = -1;
    b->exec_steps = 0;
}

}  // namespace

extern "C" {

pm_status pm_batch_workspace_size(const pm_config* cfg, int nreal, size_t* bytes) {
    PM_TRY(batch_validate(cfg, nreal, nullptr));
    if (!bytes) return fail(PM_ERR_INVALID_ARG, "null bytes");
    pm_batch b;
    b.cfg = *cfg;
    b.B = nreal;
    batch_plan(b);
    *bytes = b.total;
    return PM_OK;
}

pm_status pm_batch_init(const pm_config* cfg, int nreal, const double* boxes, void* workspace, size_t bytes,
                        void* stream, pm_batch** out) {
    if (!out) return fail(PM_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    PM_TRY(batch_validate(cfg, nreal, boxes));
    pm_batch* b = new pm_batch();
    b->cfg = *cfg;
    b->B = nreal;
    batch_plan(*b);
    if (!workspace || bytes < b->total || (uintptr_t)workspace % 256) {
        delete b;
        return fail(PM_ERR_WORKSPACE, "batch workspace too small or not 256-byte aligned");
    }
    pm_status ds = check_device();
    if (ds != PM_OK) {
        delete b;
        return ds;
    }
    b->ws = (unsigned char*)workspace;
    b->st = (cudaStream_t)stream;
    b->cosmo.omega_m = cfg->omega_m;
    b->cosmo.omega_b = cfg->omega_b;
    b->cosmo.h = cfg->h;
    b->cosmo.n_s = cfg->n_s;
    b->cosmo.sigma8 = cfg->sigma8;
    pmhost::normalise_sigma8(b->cosmo);
    const int np = cfg->np, n = cfg->nmesh;
    const size_t np3 = (size_t)np * np * np, n3 = (size_t)n * n * n, nspec = (size_t)(n / 2 + 1) * n * n;
    std::vector<double> kf(nreal), scale(nreal), amp((size_t)nreal * b->amp_len, 0.0);
    for (int r = 0; r < nreal; ++r) {
        const double box = boxes ? boxes[r] : cfg->box;
        kf[r] = 2.0 * M_PI / box;
        scale[r] = 4294967296.0 / box;
        const double V = box * box * box;
        for (int64_t n2 = 1; n2 < b->amp_len; ++n2)
            amp[(size_t)r * b->amp_len + n2] =
                std::sqrt(pmhost::power_linear(b->cosmo, kf[r] * std::sqrt((double)n2)) / V);
        pm_ctx* v = new pm_ctx();
        v->cfg = *cfg;
        v->cfg.box = box;
        v->ws = b->ws;
        v->st = b->st;
        v->n = n;
        v->np = np;
        v->np3 = (int64_t)np3;
        v->kf = kf[r];
        v->cosmo = b->cosmo;
        Layout& L = v->L;
        L.x = b->X + (size_t)r * 3 * np3 * 4;
        L.p = b->P + (size_t)r * 3 * np3 * 4;
        L.rho = b->RHO + (size_t)r * n3 * 4;
        for (int j = 0; j < 3; ++j) {
            L.spec[j] = b->SPEC[j] + (size_t)r * nspec * 8;
            L.force[j] = b->FORCE[j] + (size_t)r * n3 * 4;
        }
        L.amp = b->AMP + (size_t)r * b->amp_len * 8;
        L.bin_of = b->BIN;
        L.wtab = b->WTAB;
        L.acc = b->ACC;
        // the second and third spectrum arrays of the whole batch are the views' selection scratch
        v->scratch_off = b->SPEC[1];
        v->scratch_bytes = 2 * (size_t)nreal * nspec * 8;
        b->views.push_back(v);
    }
    std::vector<double> wtab(n / 2 + 1);
    for (int mq = 0; mq <= n / 2; ++mq) {
        const double xq = M_PI * mq / n;
        const double sq = (mq == 0) ? 1.0 : std::sin(xq) / xq;
        wtab[mq] = sq * sq;
    }
    cudaError_t e = cudaMemcpyAsync(b->at(b->AMP), amp.data(), amp.size() * 8, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->at(b->KF), kf.data(), kf.size() * 8, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->at(b->SCALE), scale.data(), scale.size() * 8, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->at(b->WTAB), wtab.data(), wtab.size() * 8, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) {
        delete b;
        return fail(PM_ERR_CUDA, std::string("pm_batch_init: ") + cudaGetErrorString(e));
    }
    *out = b;
    return PM_OK;
}

pm_status pm_batch_destroy(pm_batch* b) {
    if (b && b->exec) cudaStreamSynchronize(b->cap);
    delete b;
    return PM_OK;
}

pm_status pm_batch_context(pm_batch* b, int r, pm_ctx** view) {
    if (!b || !view || r < 0 || r >= b->B) return fail(PM_ERR_INVALID_ARG, "bad batch index");
    b->views[r]->step = b->step;
    b->views[r]->synced = b->synced;
    b->views[r]->rho_valid = false;
    // operations on a view may overwrite its slice of the batch density
    b->rho_valid = false;
    *view = b->views[r];
    return PM_OK;
}

pm_status pm_batch_ic(pm_batch* b, const uint64_t* seeds, int flags) {
    if (!b || !seeds) return fail(PM_ERR_INVALID_ARG, "null argument");
    for (int r = 0; r < b->B; ++r) PM_TRY(pm_ic_zeldovich(b->views[r], seeds[r], nullptr, flags));
    b->have_ic = true;
    b->step = 0;
    b->synced = true;
    b->rho_valid = false;
    return PM_OK;
}

pm_status pm_batch_step(pm_batch* b, int n_steps, int use_graph) {
    if (!b) return fail(PM_ERR_INVALID_ARG, "null batch");
    if (n_steps < 0) return fail(PM_ERR_INVALID_ARG, "negative step count");
    if (b->step + n_steps > b->cfg.n_steps) return fail(PM_ERR_STATE, "stepping past a_final");
    if (n_steps == 0) return PM_OK;
    if (!b->rho_valid) {
        for (int r = 0; r < b->B; ++r) PM_TRY(deposit_particles(b->views[r], b->at(b->views[r]->L.rho)));
        b->rho_valid = true;
    }
    if (!use_graph) {
        for (int k = 0; k < n_steps; ++k) PM_TRY(batch_enqueue_step(b, b->st));
        return PM_OK;
    }
    // the whole run is recorded once on the capture stream and replayed as one graph launch
    const int from = b->step;
    if (!(b->exec && b->exec_from == from && b->exec_steps == n_steps)) {
        batch_drop_graph(b);
        const bool synced0 = b->synced;
        PM_CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
        pm_status s = PM_OK;
        for (int k = 0; k < n_steps && s == PM_OK; ++k) s = batch_enqueue_step(b, b->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
        b->step = from;  // the recording only planned the steps; they run below
        b->synced = synced0;
        if (s != PM_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ce != cudaSuccess) return fail(PM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return fail(PM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        b->exec_from = from;
        b->exec_steps = n_steps;
    }
    PM_CK(cudaEventRecord(b->ev_in, b->st));
    PM_CK(cudaStreamWaitEvent(b->cap, b->ev_in, 0));
    PM_CK(cudaGraphLaunch(b->exec, b->cap));
    PM_CK(cudaEventRecord(b->ev_out, b->cap));
    PM_CK(cudaStreamWaitEvent(b->st, b->ev_out, 0));
    // advance the host-side integrator state exactly as the recorded steps did
    for (int k = 0; k < n_steps; ++k) {
        b->step += 1;
        b->synced = (b->step == b->cfg.n_steps);
    }
    return PM_OK;
}

pm_status pm_batch_set_fft(pm_batch* b, int form) {
    if (!b) return fail(PM_ERR_INVALID_ARG, "null batch");
    if (form != 0 && form != 1) return fail(PM_ERR_INVALID_ARG, "form must be 0 (separate passes) or 1 (whole planes)");
    batch_drop_graph(b);
    b->fft_form = form;
    return PM_OK;
}

pm_status pm_batch_tuning(pm_batch* b, int* chunk, int* fft_form) {
    if (!b) return fail(PM_ERR_INVALID_ARG, "null batch");
    if (chunk) *chunk = (b->chunk > 0 && b->chunk < b->B) ? b->chunk : b->B;
    if (fft_form) *fft_form = (b->fft_form == 1 && (b->cfg.nmesh == 64 || b->cfg.nmesh == 128)) ? 1 : 0;
    return PM_OK;
}

pm_status pm_batch_set_chunk(pm_batch* b, int chunk) {
    if (!b || chunk < 0 || chunk > b->B) return fail(PM_ERR_INVALID_ARG, "chunk must be in 0..nreal");
    if (chunk != b->chunk) batch_drop_graph(b);
    b->chunk = chunk;
    return PM_OK;
}

pm_status pm_batch_autotune(pm_batch* b, int* chunk_out, double* ms_out) {
    if (!b) return fail(PM_ERR_INVALID_ARG, "null batch");
    if (b->step != 0 || b->have_ic)
        return fail(PM_ERR_STATE, "autotune before pm_batch_ic (it overwrites the particles)");
    const size_t n3 = (size_t)b->cfg.nmesh * b->cfg.nmesh * b->cfg.nmesh;
    // the unperturbed lattice (x = q, p = 0) in every realisation, and its density
    PM_CK(cudaMemsetAsync(b->at(b->FORCE[0]), 0, sizeof(float) * b->B * n3, b->st));
    for (int r = 0; r < b->B; ++r) {
        pm_ctx* v = b->views[r];
        void* zero[3] = {v->at(v->L.force[0]), v->at(v->L.force[0]), v->at(v->L.force[0])};
        PM_CK(ic_place(v->at(v->L.x), v->at(v->L.p), zero, v->np, PM_FP32_FIXED, 0.0, 0.0, v->cfg.box, b->st));
    }
    for (int r = 0; r < b->B; ++r) PM_TRY(deposit_particles(b->views[r], b->at(b->views[r]->L.rho)));
    PM_CK(cudaEventRecord(b->ev_in, b->st));
    PM_CK(cudaStreamWaitEvent(b->cap, b->ev_in, 0));
    batch_drop_graph(b);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PM_CK(cudaEventCreate(&e0));
    PM_CK(cudaEventCreate(&e1));
    int best = b->B, best_form = 0;
    double best_ms = 1e300;
    pm_status st = PM_OK;
    // candidates: the form of the middle FFT passes (separate launches; whole kz planes in
    // shared memory on 64^3 and 128^3 meshes), and for each the whole batch per launch, then
    // halves down to one realisation per launch; each is one step (kick 0, drift 0: the state
    // stays the lattice) replayed from a graph
    const int nforms = (b->cfg.nmesh == 64 || b->cfg.nmesh == 128) ? 2 : 1;
    for (int form = 0; form < nforms && st == PM_OK; ++form)
    for (int c = b->B;; c = (c + 1) / 2) {
        b->chunk = c;
        b->fft_form = form;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            st = fail(PM_ERR_CUDA, "autotune: capture");
            break;
        }
        st = batch_forces_update(b, 0.0, 0.0, b->cap);
        const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
        if (st == PM_OK && ce != cudaSuccess) st = fail(PM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
        if (st == PM_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) st = fail(PM_ERR_CUDA, "autotune: instantiate");
        if (g) cudaGraphDestroy(g);
        if (st != PM_OK) break;
        float ms = 0.f;
        cudaError_t le = cudaGraphLaunch(ex, b->cap);
        if (le == cudaSuccess) le = cudaEventRecord(e0, b->cap);
        for (int k = 0; k < 3 && le == cudaSuccess; ++k) le = cudaGraphLaunch(ex, b->cap);
        if (le == cudaSuccess) le = cudaEventRecord(e1, b->cap);
        if (le == cudaSuccess) le = cudaEventSynchronize(e1);
        if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, e0, e1);
        cudaGraphExecDestroy(ex);
        if (le != cudaSuccess) {
            st = fail(PM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(le));
            break;
        }
        if (ms / 3.0 < best_ms) {
            best_ms = ms / 3.0;
            best = c;
            best_form = form;
        }
        if (c == 1) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = best;
    b->fft_form = best_form;
    b->rho_valid = false;
    if (st != PM_OK) return st;
    if (chunk_out) *chunk_out = best;
    if (ms_out) *ms_out = best_ms;
    return PM_OK;
}

pm_status pm_batch_state(pm_batch* b, int* step, double* a, int* synchronised) {
    if (!b) return fail(PM_ERR_INVALID_ARG, "null batch");
    if (step) *step = b->step;
    if (a) *a = b->a_grid(b->step);
    if (synchronised) *synchronised = b->synced ? 1 : 0;
    return PM_OK;
}

pm_status pm_batch_power(pm_batch* b, int nbins, const double* edges, int deconvolve, double* k_out, double* p_out,
                         double* nmodes_out) {
    if (!b) return fail(PM_ERR_INVALID_ARG, "null batch");
    for (int r = 0; r < b->B; ++r) {
        pm_ctx* v = nullptr;
        PM_TRY(pm_batch_context(b, r, &v));
        PM_TRY(pm_power(v, nullptr, nullptr, nbins, edges, deconvolve, k_out ? k_out + (size_t)r * nbins : nullptr,
                        p_out ? p_out + (size_t)r * nbins : nullptr,
                        nmodes_out ? nmodes_out + (size_t)r * nbins : nullptr));
    }
    return PM_OK;
}

pm_status pm_batch_bias(pm_batch* b, double fraction, int nbins, const double* edges, double k_max, int terms,
                        double* coef_out) {
    if (!b || !coef_out) return fail(PM_ERR_INVALID_ARG, "null argument");
    for (int r = 0; r < b->B; ++r) {
        pm_ctx* v = nullptr;
        PM_TRY(pm_batch_context(b, r, &v));
        void* dm = b->at(v->L.force[0]);
        void* dh = b->at(v->L.force[1]);
        PM_TRY(pm_density(v, dm));
        PM_TRY(pm_halo_proxy(v, dm, fraction, dh, nullptr));
        PM_TRY(pm_linear_bias(v, dh, dm, nbins, edges, k_max, terms, coef_out + (size_t)r * terms, nullptr, nullptr,
                              nullptr));
    }
    return PM_OK;
}

}  // extern "C"

extern "C" {

// ------------------------------------------------------------------ stateless operators
pm_status pm_cic_deposit(const void* x, int64_t count, int precision, int n, double mass, void* rho, void* stream) {
    if ((!x && count > 0) || !rho || count < 0) return fail(PM_ERR_INVALID_ARG, "null pointer or negative count");
    if (!pow2(n) || n < 2 || n > 1024) return fail(PM_ERR_INVALID_ARG, "n must be a power of two in 2..1024");
    if (precision != PM_FP32_FIXED && precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    PM_TRY(check_device());
    PM_CK(deposit(x, count, precision, n, mass, rho, (cudaStream_t)stream));
    return PM_OK;
}

pm_status pm_cic_interp(const void* field, int n, const void* x, int64_t count, int precision, void* out,
                        void* stream) {
    if (!field || (!x && count > 0) || (!out && count > 0) || count < 0)
        return fail(PM_ERR_INVALID_ARG, "null pointer or negative count");
    if (!pow2(n) || n < 2 || n > 1024) return fail(PM_ERR_INVALID_ARG, "n must be a power of two in 2..1024");
    if (precision != PM_FP32_FIXED && precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    PM_TRY(check_device());
    PM_CK(interp(field, n, x, count, precision, out, (cudaStream_t)stream));
    return PM_OK;
}

pm_status pm_cell_sort_scratch_size(int64_t count, int n, size_t* bytes) {
    if (!bytes || count < 0 || !pow2(n) || n < 2 || n > 1024) return fail(PM_ERR_INVALID_ARG, "bad arguments");
    if (count > 0xFFFFFFFFll) return fail(PM_ERR_INVALID_ARG, "count must fit in 32 bits");
    *bytes = cell_sort_scratch_bytes(count, n);
    return PM_OK;
}

pm_status pm_cell_sort(const void* x, int64_t count, int precision, int n, uint32_t* keys_out, uint32_t* order_out,
                       void* scratch, size_t scratch_bytes, void* stream) {
    size_t need = 0;
    PM_TRY(pm_cell_sort_scratch_size(count, n, &need));
    if ((!x && count > 0) || (!keys_out && count > 0)) return fail(PM_ERR_INVALID_ARG, "null pointer");
    if (order_out && (!scratch || scratch_bytes < need)) return fail(PM_ERR_WORKSPACE, "cell sort scratch too small");
    if (precision != PM_FP32_FIXED && precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    PM_TRY(check_device());
    PM_CK(cell_sort(x, count, precision, n, keys_out, order_out, scratch, (cudaStream_t)stream));
    return PM_OK;
}

pm_status pm_cell_sort_static(const void* x, int64_t count, int precision, int n, uint32_t* keys_out,
                              uint32_t* order_out, void* stream) {
    if (count < 0 || !pow2(n) || n < 2 || n > 1024) return fail(PM_ERR_INVALID_ARG, "bad arguments");
    if ((int64_t)n * n * n > PM_CELL_SORT_STATIC_MAX_CELLS || cell_sort_static_max_cells() != PM_CELL_SORT_STATIC_MAX_CELLS)
        return fail(PM_ERR_INVALID_ARG, "pm_cell_sort_static handles meshes of at most 64^3 cells; use pm_cell_sort");
    if (count > 0xFFFFFFFFll) return fail(PM_ERR_INVALID_ARG, "count must fit in 32 bits");
    if ((!x && count > 0) || (!keys_out && count > 0)) return fail(PM_ERR_INVALID_ARG, "null pointer");
    if (precision != PM_FP32_FIXED && precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    PM_TRY(check_device());
    PM_CK(cell_sort_static(x, count, precision, n, keys_out, order_out, (cudaStream_t)stream));
    return PM_OK;
}

pm_status pm_div_mode_check(const double* a, const double* d, int64_t count, double* out, void* stream) {
    if (count < 0 || (count > 0 && (!a || !d || !out))) return fail(PM_ERR_INVALID_ARG, "bad arguments");
    PM_TRY(check_device());
    PM_CK(div_mode_check(a, d, count, out, (cudaStream_t)stream));
    return PM_OK;
}

pm_status pm_fft_r2c(const void* real, void* spec, int n, int precision, void* stream) {
    if (!real || !spec) return fail(PM_ERR_INVALID_ARG, "null pointer");
    if (!pow2(n) || n < 16 || n > 1024) return fail(PM_ERR_INVALID_ARG, "n must be a power of two in 16..1024");
    if (precision != PM_FP32_FIXED && precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    PM_TRY(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    SpecOp fw;
    fw.kind = OP_FWD_STORE;
    fw.fwd = 1;
    if (precision == PM_FP64) {
        PM_CK(forward_zy<double>((const double*)real, (double2*)spec, n, 1, st));
        PM_CK(x_cols<double>((double2*)spec, nullptr, n / 2 + 1, n, fw, st));
    } else {
        PM_CK(forward_zy<float>((const float*)real, (float2*)spec, n, 1, st));
        PM_CK(x_cols<float>((float2*)spec, nullptr, n / 2 + 1, n, fw, st));
    }
    return PM_OK;
}

pm_status pm_fft_c2r(void* spec, void* real, int n, int precision, void* stream) {
    if (!real || !spec) return fail(PM_ERR_INVALID_ARG, "null pointer");
    if (!pow2(n) || n < 16 || n > 1024) return fail(PM_ERR_INVALID_ARG, "n must be a power of two in 16..1024");
    if (precision != PM_FP32_FIXED && precision != PM_FP64) return fail(PM_ERR_INVALID_ARG, "bad precision");
    PM_TRY(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    SpecOp inv;
    inv.kind = OP_INV;
    inv.fwd = 0;
    if (precision == PM_FP64) {
        PM_CK(x_cols<double>((double2*)spec, nullptr, n / 2 + 1, n, inv, st));
        PM_CK((y_rows<double, true>((double2*)spec, (int64_t)(n / 2 + 1) * n, n, st)));
        const double2* in[1] = {(double2*)spec};
        double* out[1] = {(double*)real};
        PM_CK(z_c2r<double>(in, out, 1, n, 1, 0u, 0.0, st));
    } else {
        PM_CK(x_cols<float>((float2*)spec, nullptr, n / 2 + 1, n, inv, st));
        PM_CK((y_rows<float, true>((float2*)spec, (int64_t)(n / 2 + 1) * n, n, st)));
        const float2* in[1] = {(float2*)spec};
        float* out[1] = {(float*)real};
        PM_CK(z_c2r<float>(in, out, 1, n, 1, 0u, 0.0, st));
    }
    return PM_OK;
}

}  // extern "C"
