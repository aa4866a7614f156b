// nh_api.cu -- host runtime and C-ABI of libnh (declared in include/nh.h).
//
// A handle owns the device buffers of one problem (2D grid, or a batch of 1D channels) in
// FP32 or FP64, and drives the per-stage kernels of nh_kernels.cu on the caller's stream.
// The 2D pressure solve is BiCGStab whose scalars live on the device; the host polls its
// control block every few iterations to decide when to stop.
#include "../../include/nh.h"
#include "nh_internal.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

using namespace nh;

namespace {

struct Base {
    virtual ~Base() {}
    virtual int set_state(const void* eta, const void* q1, const void* q2, const void* w,
                          const void* p, int where) = 0;
    virtual int get_state(void* eta, void* q1, void* q2, void* w, void* p, int where) = 0;
    virtual int step(double dt) = 0;
    virtual int set_relax_target(const void* eta, const void* q1, const void* q2,
                                 const void* w, const void* p, int where) = 0;
    virtual int lambda(double* lam) = 0;
    virtual int mass(double* m) = 0;
    virtual int gauges(const int* cells, int n, void* out) = 0;
    virtual int cheb_form() const = 0;   // pass form in use, -1 while timing
    virtual int debug_hyp(double dt, void* e, void* a, void* b, int where) = 0;
    virtual int debug_system(double dt, const void* x, void* rhs, void* mx, int where) = 0;
    virtual int debug_stall_copies(int block) = 0;
    virtual int profile_enable(int on) = 0;
    virtual int profile_read(nh_profile_t* out) = 0;
    virtual size_t tape_bytes() = 0;
    virtual int step_taped(double dt, void* tape) = 0;
    virtual int adjoint_step(double dt, const void* tape, void* eb, void* a1b, void* a2b,
                             void* wb, void* Hb) = 0;
};

// Intervals between recorded events (around eager launches, or between the event nodes of
// a captured step), accumulated per kernel class with their launch counts.
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Iv { cudaEvent_t a, b; int cls; long long n; };
    std::vector<Iv> iv;
    long long launches[NH_K_COUNT] = {};
    double ms[NH_K_COUNT] = {};

    ~Prof()
    {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
    cudaEvent_t next()
    {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void add(cudaEvent_t a, cudaEvent_t b, int cls, long long n) { iv.push_back({a, b, cls, n}); }
    void flush()
    {
        if (!iv.empty()) {
            cudaEventSynchronize(iv.back().b);
            for (const Iv& v : iv) {
                float t = 0.f;
                cudaEventElapsedTime(&t, v.a, v.b);
                ms[v.cls] += t;
                launches[v.cls] += v.n;
            }
        }
        iv.clear();
        used = 0;
    }
    void reset()
    {
        flush();
        for (int k = 0; k < NH_K_COUNT; ++k) { launches[k] = 0; ms[k] = 0.0; }
    }
};

}  // namespace

struct nh_handle {
    nh_grid grid;
    nh_params prm;
    cudaStream_t s = nullptr;
    std::unique_ptr<Base> impl;
    double t = 0.0, dt_last = 0.0, dt_next = 0.0;
    long long steps = 0, solver_iters = 0;
    int last_iters[2] = {0, 0};
    double last_resid[2] = {0.0, 0.0};
    int nonfinite = 0;
    int fallbacks = 0;
    long long fallback_iters = 0;
    std::string err;
};

namespace {

int fail(nh_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(nh_handle* h, cudaError_t e, const char* where)
{
    return fail(h, NH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename T>
struct Impl : Base {
    nh_handle* hd;
    Prm<T> P;
    int dim;
    size_t nc, nn;           // cells, nodes
    Launch Lc, Ln;
    Bufs<T> B{};
    std::vector<void*> allocs;
    Prof prof;
    SolveCtl* h_sctl = nullptr;   // pinned mirrors of the device control blocks
    StepCtl* h_stctl = nullptr;
    int last_solve_iters = 0;
    int last_cheb_passes = 0;
    int stall_block = -1;       // test hook (nh_debug_stall_copies): next register pass only
    RelaxZ Z{};                 // relaxation zones (Sec. 4.4); relax_on: any side has one
    bool relax_on = false;

    ~Impl() override
    {
        for (void* p : allocs) cudaFree(p);
        if (h_sctl) cudaFreeHost(h_sctl);
        if (h_sctl32) cudaFreeHost(h_sctl32);
        if (h_stctl) cudaFreeHost(h_stctl);
        for (cudaEvent_t e : vt_ev)
            if (e) cudaEventDestroy(e);
        graph_destroy();
        if (g_side) cudaStreamDestroy(g_side);
        if (g_cap) cudaStreamDestroy(g_cap);
        if (h_dt) cudaFreeHost(h_dt);
        if (h_sstat) cudaFreeHost(h_sstat);
    }

    template <typename U>
    int alloc(U** p, size_t n)
    {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(U) + 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(hd, NH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *p = static_cast<U*>(q);
        return NH_OK;
    }

    int init(nh_handle* h, const double* Hhost)
    {
        hd = h;
        const nh_grid& g = h->grid;
        const nh_params& q = h->prm;
        dim = g.dim;
        P.nx = g.nx; P.ny = g.ny;
        P.bcw = g.bc[0]; P.bce = g.bc[1]; P.bcs = g.bc[2]; P.bcn = g.bc[3];
        P.dx = (T)g.dx; P.dy = (T)(dim == 2 ? g.dy : g.dx);
        P.g = (T)q.g; P.delta = (T)q.delta; P.hdry = (T)q.hdry; P.manning = (T)q.manning_n;
        P.B1 = (T)q.B1; P.breaking = q.breaking; P.dry_zero = q.dry_zero ? 1 : 0;
        pass_variant = q.cheb_form;
        nc = (size_t)g.nx * g.ny;
        nn = dim == 2 ? (size_t)(g.nx + 1) * (g.ny + 1) : (size_t)(g.nx + 1) * g.ny;
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 148;
        // the cyclic forms are timed against each other (the same iterates), not against
        // the Jacobi forms
        cyclic = q.cheb_form < 0 && q.cheb_cyclic && !(q.eps_dp > 0.0) && dim == 2;
        if (cyclic && cheb_cyclic_forms<T>() == 1) pass_variant = cheb_pass_forms<T>();
        auto grid_for = [&](size_t n) {
            long long want = (long long)((n + 255) / 256);
            long long cap = (long long)nsm * 8;
            return (int)(want < cap ? (want > 0 ? want : 1) : cap);
        };
        Lc = {grid_for(nc), 256, h->s};
        Ln = {grid_for(nn), 256, h->s};
        const int nblk = Lc.nblk > Ln.nblk ? Lc.nblk : Ln.nblk;
        int rc = NH_OK;
#define A(ptr, n) if ((rc = alloc(&(ptr), (n))) != NH_OK) return rc
        A(B.H, nc);
        A(B.eta, nc); A(B.q1, nc); A(B.q2, nc);
        A(B.eta1, nc); A(B.q11, nc); A(B.q21, nc);
        A(B.etas, nc); A(B.q1s, nc); A(B.q2s, nc);
        if (q.breaking) { A(B.q1k, nc); A(B.q2k, nc); }
        else { B.q1k = B.q1s; B.q2k = B.q2s; }
        A(B.w, nn); A(B.p, nn); A(B.w1, nn); A(B.ws, nn);
        A(B.cC, nn); A(B.cW, nn); A(B.cE, nn); A(B.rhs, nn);
        A(B.r, nn); A(B.rh, nn);
        if (dim == 2) {
            A(B.cS, nn); A(B.cN, nn); A(B.dp, nn); A(B.palt, nn);
            A(B.ph[0], nn); A(B.ph[1], nn); A(B.v[0], nn); A(B.v[1], nn); A(B.t, nn);
        } else {
            B.cS = B.cN = B.ph[0] = B.ph[1] = B.v[0] = B.v[1] = B.t = nullptr;
            B.dp = B.palt = nullptr;
        }
        {
            size_t np = (size_t)4 * nblk + 64;
            if (dim == 2) {
                const size_t nt = 2 * cheb_tiles<T>(P) + 64;
                const size_t na = 3 * asm_tiles<T>(P) + 64;
                if (nt > np) np = nt;
                if (na > np) np = na;
            }
            A(B.partials, np);
        }
        A(B.sctl, 1);
        A(B.stctl, 1);
        for (int k = 0; k < 4; ++k) {   // k: the first natural number with k d >= L_Rel
            Z.L[k] = q.relax_width[k];
            const double d = k < 2 ? g.dx : g.dy;
            int kk = 0;
            if (Z.L[k] > 0.0)
                while ((double)kk * d < Z.L[k]) ++kk;
            Z.k[k] = kk;
            relax_on = relax_on || kk > 0;
        }
        Z.d[0] = g.dx;
        Z.d[1] = dim == 2 ? g.dy : g.dx;
        if (relax_on) {
            A(B.rz_eta, nc); A(B.rz_q1, nc); A(B.rz_w, nn); A(B.rz_p, nn);
            if (dim == 2) A(B.rz_q2, nc);
        }
        if (sizeof(T) == 8 && dim == 2 && q.nonhydrostatic &&
            q.solver == NH_SOLVER_CHEBYSHEV && q.refine_fp32 && !(q.eps_dp > 0.0)) {
            // FP32 copies of the rows and the inner solve's vectors
            float** f32[] = {&B32.cC, &B32.cW, &B32.cE, &B32.cS, &B32.cN, &B32.rhs, &B32.dp,
                             &B32.r, &B32.v[0], &B32.v[1]};
            for (float** f : f32) A(*f, nn);
            A(B32.sctl, 1);
            P32.nx = P.nx; P32.ny = P.ny;
            P32.bcw = P.bcw; P32.bce = P.bce; P32.bcs = P.bcs; P32.bcn = P.bcn;
            P32.dx = (float)P.dx; P32.dy = (float)P.dy;
            refine = true;
        }
        if (q.w_equation == NH_W_TRANSPORT) {
            // face mass fluxes: x faces [ny][nx+1] (1D: [rows][nx+1]), y faces [ny+1][nx]
            A(B.fmx, (size_t)(g.nx + 1) * g.ny);
            if (dim == 2) A(B.fmy, (size_t)g.nx * (g.ny + 1));
            A(B.wt, nn);
        }
#undef A
        cudaError_t e;
        if ((e = cudaMallocHost(&h_sctl, sizeof(SolveCtl))) != cudaSuccess) return cuda_fail(hd, e, "cudaMallocHost");
        for (cudaEvent_t& ev : vt_ev)
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(hd, e, "cudaEventCreate");
        if ((e = cudaMallocHost(&h_stctl, sizeof(StepCtl))) != cudaSuccess) return cuda_fail(hd, e, "cudaMallocHost");
        if (refine) {
            if ((e = cudaMallocHost(&h_sctl32, sizeof(SolveCtl))) != cudaSuccess)
                return cuda_fail(hd, e, "cudaMallocHost");
            cudaMemsetAsync(B32.sctl, 0, sizeof(SolveCtl), h->s);
        }
        cudaMemsetAsync(B.sctl, 0, sizeof(SolveCtl), h->s);
        cudaMemsetAsync(B.stctl, 0, sizeof(StepCtl), h->s);
        h_sctl->eps_dp = q.eps_dp;
        cudaMemcpyAsync(&B.sctl->eps_dp, &h_sctl->eps_dp, sizeof(double), cudaMemcpyHostToDevice,
                        h->s);
        // H (double on the host) -> device precision
        double* Htmp = nullptr;
        if ((e = cudaMalloc(&Htmp, nc * sizeof(double))) != cudaSuccess) {
            cudaGetLastError();
            return fail(hd, NH_ENOMEM, "cudaMalloc (H staging)");
        }
        cudaMemcpyAsync(Htmp, Hhost, nc * sizeof(double), cudaMemcpyHostToDevice, h->s);
        launch_convert_from_double<T>(Lc, Htmp, B.H, nc);
        cudaStreamSynchronize(h->s);
        cudaFree(Htmp);
        // lake at rest: eta = max(H, 0) - H, q = w = p = 0
        std::vector<double> Hv(Hhost, Hhost + nc);
        std::vector<T> eta0(nc);
        for (size_t k = 0; k < nc; ++k) eta0[k] = (T)(Hv[k] > 0.0 ? 0.0 : -Hv[k]);
        cudaMemcpyAsync(B.eta, eta0.data(), nc * sizeof(T), cudaMemcpyHostToDevice, h->s);
        launch_fill<T>(Lc, B.q1, nc, T(0));
        launch_fill<T>(Lc, B.q2, nc, T(0));
        launch_fill<T>(Ln, B.w, nn, T(0));
        launch_fill<T>(Ln, B.p, nn, T(0));
        if (relax_on) {   // absorbing target: the lake at rest
            cudaMemcpyAsync(B.rz_eta, eta0.data(), nc * sizeof(T), cudaMemcpyHostToDevice, h->s);
            launch_fill<T>(Lc, B.rz_q1, nc, T(0));
            if (B.rz_q2) launch_fill<T>(Lc, B.rz_q2, nc, T(0));
            launch_fill<T>(Ln, B.rz_w, nn, T(0));
            launch_fill<T>(Ln, B.rz_p, nn, T(0));
        }
        if ((e = cudaStreamSynchronize(h->s)) != cudaSuccess) return cuda_fail(hd, e, "nh_create");
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(hd, e, "nh_create launch");
        double lam = 0.0;
        if ((rc = lambda(&lam)) != NH_OK) return rc;
        hd->dt_next = lam > 0.0 ? hd->prm.cfl / lam : 0.0;
        return NH_OK;
    }

    // Launch f (one kernel) between two recorded events when profiling.
    template <typename F>
    void K_(int cls, F&& f)
    {
        if (!prof.on) { f(); return; }
        if (prof.used + 2 > 16384) prof.flush();
        cudaEvent_t a = prof.next(), b = prof.next();
        cudaEventRecord(a, hd->s);
        f();
        cudaEventRecord(b, hd->s);
        prof.add(a, b, cls, 1);
    }

    int profile_enable(int on) override
    {
        prof.reset();
        prof.on = on != 0;
        return NH_OK;
    }

    int profile_read(nh_profile_t* out) override
    {
        prof.flush();
        for (int k = 0; k < NH_K_COUNT; ++k) { out->launches[k] = prof.launches[k]; out->ms[k] = prof.ms[k]; }
        return NH_OK;
    }

    cudaMemcpyKind kind_in(int where) const
    {
        return where == NH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    }
    cudaMemcpyKind kind_out(int where) const
    {
        return where == NH_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    }

    int set_state(const void* eta, const void* q1, const void* q2, const void* w,
                  const void* p, int where) override
    {
        cudaStream_t s = hd->s;
        if (!eta || !q1) return fail(hd, NH_EINVAL, "nh_set_state: eta and q1 are required");
        cudaMemcpyAsync(B.eta, eta, nc * sizeof(T), kind_in(where), s);
        cudaMemcpyAsync(B.q1, q1, nc * sizeof(T), kind_in(where), s);
        if (q2) cudaMemcpyAsync(B.q2, q2, nc * sizeof(T), kind_in(where), s);
        else launch_fill<T>(Lc, B.q2, nc, T(0));
        if (w) cudaMemcpyAsync(B.w, w, nn * sizeof(T), kind_in(where), s);
        else launch_fill<T>(Ln, B.w, nn, T(0));
        if (p) cudaMemcpyAsync(B.p, p, nn * sizeof(T), kind_in(where), s);
        else launch_fill<T>(Ln, B.p, nn, T(0));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(hd, e, "nh_set_state");
        // the input must be finite (checked on the device; the rate kernel's max would
        // pass over a NaN)
        cudaMemsetAsync(&B.stctl->nonfinite, 0, sizeof(int), s);
        launch_nonfinite<T>(Lc, B.eta, nc, B.stctl);
        launch_nonfinite<T>(Lc, B.q1, nc, B.stctl);
        launch_nonfinite<T>(Lc, B.q2, nc, B.stctl);
        launch_nonfinite<T>(Ln, B.w, nn, B.stctl);
        launch_nonfinite<T>(Ln, B.p, nn, B.stctl);
        double lam = 0.0;
        int rc = lambda(&lam);
        if (rc != NH_OK) return rc;
        if (h_stctl->nonfinite)
            return fail(hd, NH_ENONFINITE, "nh_set_state: non-finite value in the input state");
        hd->dt_next = lam > 0.0 ? hd->prm.cfl / lam : 0.0;
        return NH_OK;
    }

    int get_state(void* eta, void* q1, void* q2, void* w, void* p, int where) override
    {
        cudaStream_t s = hd->s;
        if (eta) cudaMemcpyAsync(eta, B.eta, nc * sizeof(T), kind_out(where), s);
        if (q1) cudaMemcpyAsync(q1, B.q1, nc * sizeof(T), kind_out(where), s);
        if (q2) cudaMemcpyAsync(q2, B.q2, nc * sizeof(T), kind_out(where), s);
        if (w) cudaMemcpyAsync(w, B.w, nn * sizeof(T), kind_out(where), s);
        if (p) cudaMemcpyAsync(p, B.p, nn * sizeof(T), kind_out(where), s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "nh_get_state");
        return NH_OK;
    }

    int set_relax_target(const void* eta, const void* q1, const void* q2, const void* w,
                         const void* p, int where) override
    {
        if (!relax_on) return fail(hd, NH_EINVAL, "nh_set_relax_target: no relaxation zone");
        cudaStream_t s = hd->s;
        if (eta) cudaMemcpyAsync(B.rz_eta, eta, nc * sizeof(T), kind_in(where), s);
        if (q1) cudaMemcpyAsync(B.rz_q1, q1, nc * sizeof(T), kind_in(where), s);
        if (q2 && B.rz_q2) cudaMemcpyAsync(B.rz_q2, q2, nc * sizeof(T), kind_in(where), s);
        if (w) cudaMemcpyAsync(B.rz_w, w, nn * sizeof(T), kind_in(where), s);
        if (p) cudaMemcpyAsync(B.rz_p, p, nn * sizeof(T), kind_in(where), s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "nh_set_relax_target");
        return NH_OK;
    }

    int lambda(double* lam) override
    {
        launch_lambda<T>(P, Lc, B.eta, B.q1, B.q2, B.H, dim, B.partials, B.stctl);
        cudaMemcpyAsync(h_stctl, B.stctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, hd->s);
        cudaError_t e = cudaStreamSynchronize(hd->s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "lambda");
        *lam = h_stctl->lam;
        return NH_OK;
    }

    int gauges(const int* cells, int n, void* out) override
    {
        launch_gather<T>(hd->s, B.eta, cells, n, static_cast<T*>(out));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(hd, e, "nh_gauges");
        return NH_OK;
    }

    int mass(double* m) override
    {
        launch_mass<T>(P, Lc, B.eta, B.H, B.partials, B.stctl);
        cudaMemcpyAsync(h_stctl, B.stctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, hd->s);
        cudaError_t e = cudaStreamSynchronize(hd->s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "mass");
        *m = h_stctl->mass * (double)P.dx * (dim == 2 ? (double)P.dy : 1.0);
        return NH_OK;
    }

    // Chebyshev-scheduled Jacobi (temporally blocked passes); B.p is the warm start and
    // receives the solution, B.r holds the previous iterate.
    // After `passes` executed passes the iterate is in (v[0], v[1]) when passes is odd:
    // make (dp, r) hold it.
    void settle_passes(int passes)
    {
        if (passes & 1) { std::swap(B.dp, B.v[0]); std::swap(B.r, B.v[1]); }
    }

    int solve_cheb(int stage)
    {
        const int K = cheb_sweeps_per_pass<T>();
        cudaMemsetAsync(B.r, 0, nn * sizeof(T), hd->s);
        cudaMemsetAsync(B.dp, 0, nn * sizeof(T), hd->s);
        int passes_launched = 0;
        ++solves;
        int batch = last_cheb_passes > 2 ? last_cheb_passes - 1 : 4;
        for (;;) {
            for (int k = 0; k < batch; ++k) {
                int rc = 0;
                // until the faster pass form is known, alternate the two (their sweeps are
                // identical, so the solve does not depend on the choice) and time them
                const int v = pass_variant >= 0 ? pass_variant : timed_variant();
                const bool timed = pass_variant < 0 && vt_used + 2 <= kVT;
                if (timed) cudaEventRecord(vt_ev[vt_used], hd->s);
                if (timed) { vt_pass[vt_used / 2] = passes_launched; vt_solve[vt_used / 2] = solves; }
                // pass j reads buffer pair j % 2 and writes the other
                const bool odd = (passes_launched++ & 1) != 0;
                T* xa = odd ? B.v[0] : B.dp;
                T* pa = odd ? B.v[1] : B.r;
                T* xb = odd ? B.dp : B.v[0];
                T* pb = odd ? B.r : B.v[1];
                const unsigned polls = hd->prm.wait_polls > 0 ? (unsigned)hd->prm.wait_polls
                                                              : kDefaultWaitPolls;
                K_(NH_K_CHEB_PASS, [&] {
                    rc = launch_cheb_pass<T>(P, hd->s, B, xa, pa, xb, pb, B.partials, v, polls,
                                             stall_block);
                });
                stall_block = -1;   // the test hook acts on one pass
                if (timed) {
                    cudaEventRecord(vt_ev[vt_used + 1], hd->s);
                    vt_var[vt_used / 2] = v;
                    vt_used += 2;
                }
                if (rc != 0) return fail(hd, NH_ECUDA, "Chebyshev pass launch failed");
            }
            cudaMemcpyAsync(h_sctl, B.sctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, hd->s);
            cudaError_t e = cudaStreamSynchronize(hd->s);
            if (e != cudaSuccess) return cuda_fail(hd, e, "pressure solve");
            if (pass_variant < 0) {
                // passes launched after the solve converged return at once: only the timed
                // passes that ran count
                const int ran = h_sctl->done ? h_sctl->sweeps / K : passes_launched;
                for (int k = 0; k < vt_used / 2; ++k)
                    if (vt_solve[k] == solves) vt_ok[k] = vt_pass[k] < ran ? 1 : 0;
                if (vt_used >= kVT || (vt_next > 0 && solves >= 12)) choose_pass_variant();
            }
            if (h_sctl->status == 6 || h_sctl->status == 7) {
                hd->last_iters[stage] = h_sctl->sweeps;
                return fail(hd, NH_ETIMEOUT,
                            h_sctl->status == 6
                                ? "Chebyshev pass: a wait for staged copies ran out of polls "
                                  "(the copies issued were drained; the solve was abandoned)"
                                : "Chebyshev pass: a wait for staged copies ran out of polls "
                                  "and so did the drain of the copies in flight");
            }
            if (h_sctl->status == 4) return fallback(stage, false);   // not diagonally dominant
            if (!h_sctl->done) { batch = 2; continue; }
            settle_passes(h_sctl->sweeps / K);
            if (h_sctl->status == 5) {
                // stalled (cheb_finish_stall: the rounding floor of the precision, or a
                // spectrum the Gershgorin interval does not describe): continue with
                // BiCGStab from the current dp (under criterion (32) only a residual that
                // no longer falls at all counts as stalled)
                last_cheb_passes = h_sctl->sweeps / K;
                if (accept_stall) {   // adjoint solves: the precision's floor is accepted
                    hd->solver_iters += h_sctl->sweeps;
                    hd->last_iters[stage] = h_sctl->sweeps;
                    hd->last_resid[stage] =
                        h_sctl->bdb > 0.0 ? std::sqrt(h_sctl->rr / h_sctl->bdb) : 0.0;
                    return NH_OK;
                }
                return fallback(stage, true);
            }
            break;
        }
        const int sweeps = h_sctl->sweeps;
        last_cheb_passes = sweeps / K;
        hd->solver_iters += sweeps;
        hd->last_iters[stage] = sweeps;
        hd->last_resid[stage] = h_sctl->bdb > 0.0 ? std::sqrt(h_sctl->rr / h_sctl->bdb) : 0.0;
        if (h_sctl->status != 1)
            return fail(hd, NH_ENOCONV,
                        "Chebyshev solve stopped after " + std::to_string(sweeps) +
                            " sweeps with scaled residual " +
                            std::to_string(hd->last_resid[stage]));
        return NH_OK;
    }

    // A Chebyshev solve handed over to BiCGStab (counted in the statistics).
    int fallback(int stage, bool keep_dp)
    {
        const long long before = hd->solver_iters;
        const int rc = solve2d(stage, keep_dp);
        hd->fallbacks += 1;
        hd->fallback_iters += hd->solver_iters - before;
        return rc;
    }

    // BiCGStab on the correction system M dp = r0 (from dp = 0, or from the current dp when
    // continuing a stalled Chebyshev solve).
    int solve2d(int stage, bool keep_dp = false)
    {
        const nh_params& q = hd->prm;
        if (!keep_dp) cudaMemsetAsync(B.dp, 0, nn * sizeof(T), hd->s);
        K_(NH_K_SOLVE_INIT, [&] { launch_bicg_init<T>(P, Ln, B, B.partials); });
        int launched = 0, restarts = 0;
        int batch = last_solve_iters > 2 ? last_solve_iters - 1 : 2;
        int status = 0;
        for (;;) {
            for (int k = 0; k < batch; ++k) {
                const int par = launched & 1;
                K_(NH_K_BICG_A, [&] { launch_bicg_phase<T>(P, Ln, B, par, 0, B.partials); });
                K_(NH_K_BICG_B, [&] { launch_bicg_phase<T>(P, Ln, B, par, 1, B.partials); });
                K_(NH_K_BICG_C, [&] { launch_bicg_phase<T>(P, Ln, B, par, 2, B.partials); });
                ++launched;
            }
            cudaMemcpyAsync(h_sctl, B.sctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, hd->s);
            cudaError_t e = cudaStreamSynchronize(hd->s);
            if (e != cudaSuccess) return cuda_fail(hd, e, "pressure solve");
            if (h_sctl->done) {
                status = h_sctl->status;
                if (status == 3 && restarts < 8 && h_sctl->iter < q.max_iter) {
                    ++restarts;
                    K_(NH_K_SOLVE_INIT, [&] { launch_bicg_init<T>(P, Ln, B, B.partials); });
                    launched = 0;
                    batch = 2;
                    continue;
                }
                break;
            }
            batch = 2;
        }
        const int it = h_sctl->iter;
        last_solve_iters = it;
        hd->solver_iters += it;
        hd->last_iters[stage] = it;
        hd->last_resid[stage] = h_sctl->bb > 0.0 ? std::sqrt(h_sctl->rr / h_sctl->bb) : 0.0;
        if (status != 1)
            return fail(hd, NH_ENOCONV,
                        "pressure solve stopped after " + std::to_string(it) +
                            " iterations with relative residual " +
                            std::to_string(hd->last_resid[stage]) +
                            (status == 3 ? " (breakdown)" : " (iteration cap)"));
        return NH_OK;
    }

    int stage2d(int s, T dt)
    {
        const nh_params& q = hd->prm;
        const T a = s == 0 ? T(0) : T(0.5), b = s == 0 ? T(1) : T(0.5);
        const T de = b * dt;
        const T* ein = s == 0 ? B.eta : B.eta1;
        const T* ain = s == 0 ? B.q1 : B.q11;
        const T* bin = s == 0 ? B.q2 : B.q21;
        const T* win = s == 0 ? B.w : B.w1;
        T* eo = s == 0 ? B.eta1 : B.eta;
        T* ao = s == 0 ? B.q11 : B.q1;
        T* bo = s == 0 ? B.q21 : B.q2;
        T* wo = s == 0 ? B.w1 : B.w;
        const bool wt = B.wt != nullptr;   // w equation (hw)_t + div(hw u) = p
        K_(NH_K_HYPERBOLIC, [&] {
            launch_hyp2d<T>(P, Lc, ein, ain, bin, B.eta, B.q1, B.q2, B.H, a, b, dt, B.etas,
                            B.q1s, B.q2s, B.stctl, B.fmx, B.fmy);
        });
        // transported w* (the assembly then takes it as it is: a = 0, b = 1)
        if (wt)
            K_(NH_K_W_TRANSPORT, [&] {
                launch_wtrans2d<T>(P, Ln, B.eta, ein, B.etas, B.H, B.w, win, B.fmx, B.fmy, a,
                                   b, dt, B.wt);
            });
        // the breaking terms (q* -> q**) run inside the assembly
        K_(NH_K_ASSEMBLY, [&] {
            launch_asm2d<T>(P, Ln, B, wt ? B.wt : win, wt ? B.wt : B.w, wt ? T(0) : a,
                            wt ? T(1) : b, de, q.nonhydrostatic ? 1 : 0,
                            q.nonhydrostatic ? 1 : 0, q.tol * q.tol, q.max_iter,
                            q.solver == NH_SOLVER_CHEBYSHEV ? cheb_sweeps_per_pass<T>() : 0,
                            B.partials, B.sctl, 1);
        });
        int rc = NH_OK;
        if (q.nonhydrostatic)
            rc = q.solver == NH_SOLVER_CHEBYSHEV ? (refine ? solve_refine(s) : solve_cheb(s))
                                                 : solve2d(s, false);
        K_(NH_K_CORRECTION, [&] {
            launch_corr2d<T>(P, Ln, B, B.q1k, B.q2k, de, q.nonhydrostatic ? 1 : 0, eo, ao, bo,
                             wo, s == 1 ? 1 : 0, B.partials, B.stctl);
        });
        std::swap(B.p, B.palt);
        return rc;
    }

    // ---- steps captured as CUDA graphs (2D; Chebyshev solver once its pass form is known,
    // or the hydrostatic step alone).  One graph holds a whole step: the step's dt is copied
    // from pinned host memory by its first node, the kernels read it from device memory,
    // the pressure solve is a conditional WHILE node over pairs of passes (its condition
    // kernel reads the solve's done flag), a stalled or not diagonally dominant solve
    // continues in a second WHILE node of BiCGStab iterations, and the last nodes copy the
    // step's control blocks to pinned host memory: the host waits once per step, on the
    // step's end, and polls nothing.  Results are those of the eagerly launched step bit for
    // bit (same kernels, same arguments; the iterate of a solve that ends on an odd pass is
    // read from its buffer by the correction instead of swapping pointers on the host).
    cudaGraph_t g_graph = nullptr;
    cudaGraphExec_t g_exec = nullptr;
    cudaStream_t g_cap = nullptr;    // the step is captured on this stream (the caller's may
                                     // be the legacy default stream, which cannot capture)
                                     // and launched on the caller's
    cudaStream_t g_side = nullptr;   // capture of the WHILE bodies
    T* g_p = nullptr;                // B.p when captured (the p / palt roles)
    bool g_prof = false;             // captured with event nodes (profiling)
    bool g_failed = false;           // a capture failed: the handle stays eager
    double* d_dt = nullptr;          // the step's dt (device) and its pinned source
    double* h_dt = nullptr;
    unsigned* d_loopc = nullptr;     // [pass pairs, BiCGStab pairs] of the running stage
    SolveStat* d_sstat = nullptr;    // per stage, and pinned copies written by the graph
    SolveStat* h_sstat = nullptr;
    std::vector<cudaGraphNode_t> g_evnodes;   // event record nodes (profiling)
    struct GIv { int a, b, cls, stage; };      // interval between event nodes a and b
    std::vector<GIv> g_iv;
    bool capturing = false;

    bool graph_mode() const
    {
        const nh_params& q = hd->prm;
        // (after one eager step: the kernels' one-time attribute and occupancy set-up runs
        // outside the capture)
        return q.capture && dim == 2 && !g_failed && stall_block < 0 && eager_steps > 0 &&
               !refine &&
               (!q.nonhydrostatic || (q.solver == NH_SOLVER_CHEBYSHEV && pass_variant >= 0));
    }

    void graph_destroy()
    {
        if (g_exec) cudaGraphExecDestroy(g_exec);
        if (g_graph) cudaGraphDestroy(g_graph);
        g_exec = nullptr;
        g_graph = nullptr;
        g_evnodes.clear();
        g_iv.clear();
    }

    // an event record node (profiling), returned as its index
    template <typename Chk>
    int gev(cudaStream_t st, Chk& chk)
    {
        if (!g_prof) return -1;
        cudaEvent_t e = prof.next();
        chk(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        chk(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd));
        g_evnodes.push_back(nd ? deps[0] : nullptr);
        return (int)g_evnodes.size() - 1;
    }

    // WHILE node on the capturing stream: `pre` (on that stream) sets the condition before
    // the first iteration; `body` is captured into the node's body graph on g_side.
    template <typename Chk, typename Pre, typename Body>
    void add_while(Chk& chk, Pre&& pre, Body&& body)
    {
        cudaStream_t st = hd->s;
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        chk(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h = 0;
        chk(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        pre(st, h);
        chk(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
        // (the params union has no default constructor: zeroed storage)
        alignas(cudaGraphNodeParams) unsigned char npb[sizeof(cudaGraphNodeParams)] = {};
        cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npb);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        chk(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
        if (!node) return;
        cudaGraph_t bodyg = np.conditional.phGraph_out[0];
        chk(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                cudaStreamSetCaptureDependencies));
        chk(cudaStreamBeginCaptureToGraph(g_side, bodyg, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
        body(g_side, h);
        chk(cudaGetLastError());
        cudaGraph_t bout = nullptr;
        chk(cudaStreamEndCapture(g_side, &bout));
    }

    // One stage of a captured step (the graph's share of stage2d and solve_cheb).
    template <typename Chk>
    void stage2d_capture(int s, Chk& chk)
    {
        const nh_params& q = hd->prm;
        cudaStream_t st = hd->s;
        const T a = s == 0 ? T(0) : T(0.5), b = s == 0 ? T(1) : T(0.5);
        const T* ein = s == 0 ? B.eta : B.eta1;
        const T* ain = s == 0 ? B.q1 : B.q11;
        const T* bin = s == 0 ? B.q2 : B.q21;
        const T* win = s == 0 ? B.w : B.w1;
        T* eo = s == 0 ? B.eta1 : B.eta;
        T* ao = s == 0 ? B.q11 : B.q1;
        T* bo = s == 0 ? B.q21 : B.q2;
        T* wo = s == 0 ? B.w1 : B.w;
        const bool wt = B.wt != nullptr;
        const int K = cheb_sweeps_per_pass<T>();
        auto iv = [&](int e0, int e1, int cls) {
            if (e0 >= 0 && e1 >= 0) g_iv.push_back({e0, e1, cls, s});
        };
        chk(cudaMemsetAsync(d_loopc, 0, 2 * sizeof(unsigned), st));
        const int e0 = gev(st, chk);
        launch_hyp2d<T>(P, Lc, ein, ain, bin, B.eta, B.q1, B.q2, B.H, a, b, T(0), B.etas, B.q1s,
                        B.q2s, B.stctl, B.fmx, B.fmy, d_dt);
        int e1 = gev(st, chk);
        iv(e0, e1, NH_K_HYPERBOLIC);
        if (wt) {
            launch_wtrans2d<T>(P, Ln, B.eta, ein, B.etas, B.H, B.w, win, B.fmx, B.fmy, a, b,
                               T(0), B.wt, d_dt);
            const int ew = gev(st, chk);
            iv(e1, ew, NH_K_W_TRANSPORT);
            e1 = ew;
        }
        launch_asm2d<T>(P, Ln, B, wt ? B.wt : win, wt ? B.wt : B.w, wt ? T(0) : a,
                        wt ? T(1) : b, T(0), q.nonhydrostatic ? 1 : 0, q.nonhydrostatic ? 1 : 0,
                        q.tol * q.tol, q.max_iter, q.nonhydrostatic ? K : 0, B.partials, B.sctl,
                        1, d_dt, b);
        const int e2 = gev(st, chk);
        iv(e1, e2, NH_K_ASSEMBLY);
        int e3 = e2;
        if (q.nonhydrostatic) {
            chk(cudaMemsetAsync(B.r, 0, nn * sizeof(T), st));
            chk(cudaMemsetAsync(B.dp, 0, nn * sizeof(T), st));
            const unsigned polls = q.wait_polls > 0 ? (unsigned)q.wait_polls : kDefaultWaitPolls;
            const unsigned pair_cap = (unsigned)(q.max_iter / (2 * K) + 2);
            int prc = 0;
            // WHILE (solve not done) { pass (dp, r) -> (v0, v1); pass (v0, v1) -> (dp, r) }
            add_while(chk,
                      [&](cudaStream_t ps, cudaGraphConditionalHandle h) {
                          launch_loop_cond(ps, h, B.sctl, d_loopc, pair_cap, 0);
                      },
                      [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
                          prc |= launch_cheb_pass<T>(P, bs, B, B.dp, B.r, B.v[0], B.v[1],
                                                     B.partials, pass_variant, polls, -1);
                          prc |= launch_cheb_pass<T>(P, bs, B, B.v[0], B.v[1], B.dp, B.r,
                                                     B.partials, pass_variant, polls, -1);
                          launch_loop_cond(bs, h, B.sctl, d_loopc, pair_cap, 1);
                      });
            if (prc != 0) chk(cudaErrorLaunchFailure);
            // fallback: BiCGStab from the passes' iterate (moved to dp when odd)
            launch_fb_begin(st, B.sctl);
            Launch Lns = Ln;
            launch_settle_fb<T>(Lns, B.sctl, B.v[0], B.dp, nn, K);
            launch_bicg_init<T>(P, Ln, B, B.partials, 1);
            const unsigned bicg_cap = (unsigned)(q.max_iter / 2 + 2);
            add_while(chk,
                      [&](cudaStream_t ps, cudaGraphConditionalHandle h) {
                          launch_loop_cond(ps, h, B.sctl, d_loopc + 1, bicg_cap, 0);
                      },
                      [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
                          Launch Lb = Ln;
                          Lb.s = bs;
                          for (int par = 0; par < 2; ++par)
                              for (int ph = 0; ph < 3; ++ph)
                                  launch_bicg_phase<T>(P, Lb, B, par, ph, B.partials);
                          launch_loop_cond(bs, h, B.sctl, d_loopc + 1, bicg_cap, 1);
                      });
            launch_solve_stats(st, B.sctl, d_loopc, d_sstat + s);
            e3 = gev(st, chk);
            iv(e2, e3, NH_K_CHEB_PASS);
        }
        launch_corr2d<T>(P, Ln, B, B.q1k, B.q2k, T(0), q.nonhydrostatic ? 1 : 0, eo, ao, bo, wo,
                         s == 1 ? 1 : 0, B.partials, B.stctl, d_dt, b,
                         q.nonhydrostatic ? B.v[0] : nullptr);
        const int e4 = gev(st, chk);
        iv(e3, e4, NH_K_CORRECTION);
        std::swap(B.p, B.palt);
    }

    int capture()
    {
        cudaError_t e;
        if (!g_side && (e = cudaStreamCreateWithFlags(&g_side, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(hd, e, "cudaStreamCreate");
        if (!g_cap && (e = cudaStreamCreateWithFlags(&g_cap, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(hd, e, "cudaStreamCreate");
        if (!h_dt) {
            int rc = NH_OK;
            if ((rc = alloc(&d_dt, 1)) != NH_OK || (rc = alloc(&d_loopc, 2)) != NH_OK ||
                (rc = alloc(&d_sstat, 2)) != NH_OK)
                return rc;
            if ((e = cudaMallocHost(&h_dt, sizeof(double))) != cudaSuccess ||
                (e = cudaMallocHost(&h_sstat, 2 * sizeof(SolveStat))) != cudaSuccess)
                return cuda_fail(hd, e, "cudaMallocHost");
        }
        graph_destroy();
        g_prof = prof.on;
        if (g_prof) prof.flush();
        g_p = B.p;
        // every launch of the step goes to the capture stream meanwhile
        const cudaStream_t user = hd->s;
        hd->s = g_cap;
        Lc.s = Ln.s = g_cap;
        cudaStream_t st = g_cap;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            cudaGetLastError();
            hd->s = Lc.s = Ln.s = user;
            return cuda_fail(hd, e, "cudaStreamBeginCapture");
        }
        capturing = true;
        cudaError_t first = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (first == cudaSuccess && x != cudaSuccess) first = x; };
        chk(cudaMemcpyAsync(d_dt, h_dt, sizeof(double), cudaMemcpyHostToDevice, st));
        chk(cudaMemsetAsync(&B.stctl->clamped, 0, sizeof(int), st));
        for (int s = 0; s < 2; ++s) stage2d_capture(s, chk);
        if (relax_on) {   // zones after the step, then the Eq. (23) rate of the result
            const int r0 = gev(st, chk);
            launch_relax<T>(P, Ln, Z, dim, B.eta, B.q1, B.q2, B.w, B.p, B.H, B.rz_eta, B.rz_q1,
                            B.rz_q2, B.rz_w, B.rz_p);
            launch_lambda<T>(P, Lc, B.eta, B.q1, B.q2, B.H, dim, B.partials, B.stctl);
            const int r1 = gev(st, chk);
            if (r0 >= 0) g_iv.push_back({r0, r1, NH_K_RELAX, -1});
        }
        chk(cudaMemcpyAsync(h_stctl, B.stctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, st));
        chk(cudaMemcpyAsync(h_sstat, d_sstat, 2 * sizeof(SolveStat), cudaMemcpyDeviceToHost, st));
        chk(cudaGetLastError());
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(st, &graph);
        capturing = false;
        hd->s = Lc.s = Ln.s = user;
        if (first == cudaSuccess) first = e;
        if (first == cudaSuccess) first = cudaGraphInstantiate(&g_exec, graph, 0);
        g_graph = graph;
        if (g_prof) prof.used = 0;   // the capture's events only stand for nodes
        if (first != cudaSuccess) {
            cudaGetLastError();
            graph_destroy();
            return cuda_fail(hd, first, "step graph");
        }
        return NH_OK;
    }

    int step_graph(double dtd)
    {
        if (g_exec && (g_p != B.p || g_prof != prof.on)) graph_destroy();
        if (!g_exec) {
            const int rc = capture();
            if (rc != NH_OK) {   // stay eager (the message of the failure is kept)
                g_failed = true;
                return step_impl(dtd, nullptr);
            }
        }
        *h_dt = dtd;
        std::vector<cudaEvent_t> ev;
        if (g_prof) {
            if (prof.used + g_evnodes.size() > 16384) prof.flush();
            for (cudaGraphNode_t nd : g_evnodes) {
                cudaEvent_t x = prof.next();
                const cudaError_t es = cudaGraphExecEventRecordNodeSetEvent(g_exec, nd, x);
                if (es != cudaSuccess) return cuda_fail(hd, es, "profiling event of a step graph");
                ev.push_back(x);
            }
        }
        cudaError_t e = cudaGraphLaunch(g_exec, hd->s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "cudaGraphLaunch");
        if ((e = cudaStreamSynchronize(hd->s)) != cudaSuccess) return cuda_fail(hd, e, "nh_step");
        const nh_params& q = hd->prm;
        const int K = cheb_sweeps_per_pass<T>();
        int rc = NH_OK;
        for (int s = 0; s < 2 && q.nonhydrostatic; ++s) {
            const SolveStat& S = h_sstat[s];
            const int it = S.fb ? S.iter : S.sweeps;
            hd->solver_iters += it;
            hd->last_iters[s] = it;
            last_cheb_passes = S.sweeps / K;
            if (S.fb) {
                hd->fallbacks += 1;
                hd->fallback_iters += it;
                hd->last_resid[s] = S.bb > 0.0 ? std::sqrt(S.rr / S.bb) : 0.0;
            } else {
                hd->last_resid[s] = S.bdb > 0.0 ? std::sqrt(S.rr / S.bdb) : 0.0;
            }
            if (rc == NH_OK && (S.status == 6 || S.status == 7))
                rc = fail(hd, NH_ETIMEOUT, "Chebyshev pass: a wait for staged copies ran out "
                                           "of polls (the solve was abandoned)");
            else if (rc == NH_OK && S.status != 1)
                rc = fail(hd, NH_ENOCONV, "pressure solve of stage " + std::to_string(s + 1) +
                                              " stopped with status " + std::to_string(S.status) +
                                              " after " + std::to_string(it) + " iterations");
        }
        if (g_prof)
            for (const GIv& v : g_iv) {
                long long n = 1;
                if (v.cls == NH_K_CHEB_PASS) n = h_sstat[v.stage].passes;
                if (v.cls == NH_K_RELAX) n = 2;
                prof.add(ev[v.a], ev[v.b], v.cls, n);
            }
        hd->dt_next = h_stctl->lam > 0.0 ? hd->prm.cfl / h_stctl->lam : 0.0;
        if (h_stctl->nonfinite) {
            hd->nonfinite = 1;
            return fail(hd, NH_ENONFINITE, "non-finite value in the state");
        }
        return rc;
    }

    int stage1d(int s, T dt)
    {
        const nh_params& q = hd->prm;
        const T a = s == 0 ? T(0) : T(0.5), b = s == 0 ? T(1) : T(0.5);
        const T de = b * dt;
        const T* ein = s == 0 ? B.eta : B.eta1;
        const T* ain = s == 0 ? B.q1 : B.q11;
        const T* win = s == 0 ? B.w : B.w1;
        T* eo = s == 0 ? B.eta1 : B.eta;
        T* ao = s == 0 ? B.q11 : B.q1;
        T* wo = s == 0 ? B.w1 : B.w;
        const bool wt = B.wt != nullptr;   // w equation (hw)_t + (hw u)_x = p
        K_(NH_K_HYPERBOLIC, [&] {
            launch_hyp1d<T>(P, Lc, ein, ain, B.eta, B.q1, B.H, a, b, dt, B.etas, B.q1s, B.stctl,
                            B.fmx);
        });
        if (wt)
            K_(NH_K_W_TRANSPORT, [&] {
                launch_wtrans1d<T>(P, Ln, B.eta, ein, B.etas, B.H, B.w, win, B.fmx, a, b, dt,
                                   B.wt);
            });
        if (q.breaking)
            K_(NH_K_BREAKING, [&] { launch_break1d<T>(P, Lc, B.etas, B.q1s, B.H, de, B.q1k); });
        K_(NH_K_ASSEMBLY, [&] {
            launch_asm1d<T>(P, Ln, B, B.q1s, B.q1k, wt ? B.wt : win, wt ? B.wt : B.w,
                            wt ? T(0) : a, wt ? T(1) : b, de);
        });
        if (q.nonhydrostatic) {
            int trc = 0;
            K_(NH_K_TRIDIAG, [&] { trc = launch_tridiag1d<T>(P, hd->s, B, B.p); });
            if (trc != 0) return fail(hd, NH_ECUDA, "tridiagonal solve launch failed");
            hd->last_iters[s] = 1;
        }
        K_(NH_K_CORRECTION, [&] {
            launch_corr1d<T>(P, Ln, B, B.q1k, de, q.nonhydrostatic ? 1 : 0, eo, ao, wo,
                             s == 1 ? 1 : 0, B.partials, B.stctl);
        });
        return NH_OK;
    }

    int step(double dtd) override
    {
        return graph_mode() ? step_graph(dtd) : step_impl(dtd, nullptr);
    }

    // ---- tape of one step for the adjoint: U^n, U1, the stage-1 q* and p, eta^{n+1}, the
    // stage-2 q* and p (15 arrays, each starting on a 256-byte boundary)
    size_t padded(size_t n) const
    {
        const size_t al = 256 / sizeof(T);
        return (n + al - 1) / al * al;
    }
    static bool tape_is_node(int k) { return k == 3 || k == 7 || k == 10 || k == 14; }
    T* tape_at(void* tape, int k) const
    {
        size_t off = 0;
        for (int j = 0; j < k; ++j) off += padded(tape_is_node(j) ? nn : nc);
        return static_cast<T*>(tape) + off;
    }
    size_t tape_bytes() override { return (11 * padded(nc) + 4 * padded(nn)) * sizeof(T); }
    void tcopy(void* tape, int k, const T* src)
    {
        cudaMemcpyAsync(tape_at(tape, k), src, (tape_is_node(k) ? nn : nc) * sizeof(T),
                        cudaMemcpyDeviceToDevice, hd->s);
    }
    int step_taped(double dtd, void* tape) override { return step_impl(dtd, tape); }

    int eager_steps = 0;
    int step_impl(double dtd, void* tape)
    {
        ++eager_steps;
        const T dt = (T)dtd;
        cudaMemsetAsync(&B.stctl->clamped, 0, sizeof(int), hd->s);
        if (tape) { tcopy(tape, 0, B.eta); tcopy(tape, 1, B.q1); tcopy(tape, 2, B.q2); tcopy(tape, 3, B.w); }
        int rc1 = dim == 2 ? stage2d(0, dt) : stage1d(0, dt);
        if (rc1 != NH_OK && rc1 != NH_ENOCONV) return rc1;
        if (tape) {
            tcopy(tape, 4, B.eta1); tcopy(tape, 5, B.q11); tcopy(tape, 6, B.q21); tcopy(tape, 7, B.w1);
            tcopy(tape, 8, B.q1k); tcopy(tape, 9, B.q2k); tcopy(tape, 10, B.p);
        }
        int rc2 = dim == 2 ? stage2d(1, dt) : stage1d(1, dt);
        if (rc2 != NH_OK && rc2 != NH_ENOCONV) return rc2;
        if (relax_on) {   // zones after the step, then the Eq. (23) rate of the result
            K_(NH_K_RELAX, [&] {
                launch_relax<T>(P, Ln, Z, dim, B.eta, B.q1, B.q2, B.w, B.p, B.H, B.rz_eta,
                                B.rz_q1, B.rz_q2, B.rz_w, B.rz_p);
            });
            K_(NH_K_RELAX, [&] {
                launch_lambda<T>(P, Lc, B.eta, B.q1, B.q2, B.H, dim, B.partials, B.stctl);
            });
        }
        if (tape) {
            tcopy(tape, 11, B.eta); tcopy(tape, 12, B.q1k); tcopy(tape, 13, B.q2k);
            tcopy(tape, 14, B.p);
        }
        cudaMemcpyAsync(h_stctl, B.stctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, hd->s);
        cudaError_t e = cudaStreamSynchronize(hd->s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "nh_step");
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(hd, e, "nh_step launch");
        hd->dt_next = h_stctl->lam > 0.0 ? hd->prm.cfl / h_stctl->lam : 0.0;
        if (h_stctl->nonfinite) {
            hd->nonfinite = 1;
            return fail(hd, NH_ENONFINITE, "non-finite value in the state");
        }
        return rc1 != NH_OK ? rc1 : rc2;
    }

    // ---- adjoint of one step (reverse of the two stages; see nh_adjoint.cu)
    T *aEs = nullptr, *aA1 = nullptr, *aA2 = nullptr, *aHh = nullptr, *aSb = nullptr;
    T *aGh = nullptr, *aGe = nullptr, *aGu = nullptr, *aGv = nullptr;
    T *aE1 = nullptr, *aQ11 = nullptr, *aQ21 = nullptr, *aW1 = nullptr;
    T *aE0 = nullptr, *aQ10 = nullptr, *aQ20 = nullptr, *aW0 = nullptr;
    T *tW = nullptr, *tE = nullptr, *tS = nullptr, *tN = nullptr;

    int adjoint_alloc()
    {
        if (aEs) return NH_OK;
        int rc = NH_OK;
#define A(ptr, n) if ((rc = alloc(&(ptr), (n))) != NH_OK) return rc
        A(aEs, nc); A(aA1, nc); A(aA2, nc); A(aHh, nc); A(aSb, nc);
        A(aGh, nc); A(aGe, nc); A(aGu, nc); A(aGv, nc);
        A(aE1, nc); A(aQ11, nc); A(aQ21, nc); A(aW1, nn);
        A(aE0, nc); A(aQ10, nc); A(aQ20, nc); A(aW0, nn);
        A(tW, nn); A(tE, nn); A(tS, nn); A(tN, nn);
#undef A
        return NH_OK;
    }

    // Transposed solve M^T lambda = B.rhs into B.dp with the handle's solver.
    int solve_transposed(int stage)
    {
        const nh_params& q = hd->prm;
        const int cheb = q.solver == NH_SOLVER_CHEBYSHEV;
        K_(NH_K_ADJ_ASSEMBLY, [&] {
            launch_transpose<T>(P, Ln, B, B.rhs, tW, tE, tS, tN, q.tol * q.tol, q.max_iter,
                                cheb ? cheb_sweeps_per_pass<T>() : 0);
        });
        std::swap(B.cW, tW); std::swap(B.cE, tE); std::swap(B.cS, tS); std::swap(B.cN, tN);
        accept_stall = true;
        const int rc = cheb ? solve_cheb(stage) : solve2d(stage, false);
        accept_stall = false;
        std::swap(B.cW, tW); std::swap(B.cE, tE); std::swap(B.cS, tS); std::swap(B.cN, tN);
        return rc;
    }

    // Reverse of stage s (0: a = 0, b = 1; 1: a = b = 1/2).  in*: the stage's input state,
    // es, q1s, q2s, ps: its eta*, q*, p; o*: adjoint of its output (read); in*_b: adjoint of
    // the input (assigned when s == 1, accumulated when s == 0); base adjoint accumulated
    // into aE0, aQ10, aQ20, aW0.
    int adjoint_stage(int s, T dt, const T* ein, const T* q1in, const T* q2in, const T* win,
                      const T* wbase, const T* es, const T* q1s, const T* q2s, const T* ps,
                      const T* eob, const T* a1ob, const T* a2ob, const T* wob, T* ein_b,
                      T* a1in_b, T* a2in_b, T* win_b, T* Hb)
    {
        const nh_params& q = hd->prm;
        const T a = s == 0 ? T(0) : T(0.5), b = s == 0 ? T(1) : T(0.5);
        const T de = b * dt;
        // rows of the stage's system and w* (into B.ws), exactly as in the forward
        Bufs<T> D = B;
        D.etas = const_cast<T*>(es); D.q1s = const_cast<T*>(q1s); D.q2s = const_cast<T*>(q2s);
        D.q1k = D.q1s; D.q2k = D.q2s;
        K_(NH_K_ASSEMBLY, [&] {
            launch_asm2d<T>(P, Ln, D, win, wbase, a, b, de, 1, 0, 0.0, 1, 0, B.partials, B.sctl);
        });
        // p_bar, then lambda = M^-T p_bar
        K_(NH_K_ADJ_CORRECTION, [&] { launch_adj_pbar<T>(P, Ln, es, B.H, a1ob, a2ob, wob, de, B.rhs); });
        int rc = solve_transposed(s);
        if (rc != NH_OK) return rc;
        for (T* z : {aEs, aA1, aA2, aHh, aSb, aGh, aGe, aGu, aGv})
            cudaMemsetAsync(z, 0, nc * sizeof(T), hd->s);
        const double scale = 8.0 * (double)P.dx * (double)P.dy / (double)de;
        K_(NH_K_ADJ_ASSEMBLY, [&] {
            launch_adj_node<T>(P, Ln, es, B.H, q1s, q2s, B.ws, ps, B.dp, wob, scale, (double)de,
                               (double)a, (double)b, s == 1 ? 1 : 0, aHh, aSb, aA1, aA2, win_b,
                               aW0);
        });
        K_(NH_K_ADJ_CORRECTION, [&] {
            launch_adj_cell_corr<T>(P, Lc, es, B.H, ps, eob, a1ob, a2ob, de, aEs, aHh, aSb, aA1,
                                    aA2);
        });
        K_(NH_K_ADJ_CORRECTION, [&] { launch_adj_combine<T>(Lc, (long long)nc, aEs, aHh, aSb, Hb); });
        K_(NH_K_ADJ_HYPERBOLIC, [&] {
            launch_adj_face<T>(P, Lc, ein, q1in, q2in, B.H, aEs, aA1, aA2, b, dt,
                               q.adjoint_frozen_limiter, aGh, aGe, aGu, aGv);
        });
        K_(NH_K_ADJ_HYPERBOLIC, [&] {
            launch_adj_cell_hyp<T>(P, Lc, ein, q1in, q2in, B.H, aEs, aA1, aA2, aGh, aGe, aGu, aGv,
                                   a, b, s == 1 ? 1 : 0, ein_b, a1in_b, a2in_b, aE0, aQ10, aQ20,
                                   Hb);
        });
        (void)q;
        return NH_OK;
    }

    int adjoint_step(double dtd, const void* tape, void* ebv, void* a1bv, void* a2bv, void* wbv,
                     void* Hbv) override
    {
        const nh_params& q = hd->prm;
        if (dim != 2 || !q.nonhydrostatic || q.breaking || q.manning_n > 0.0 ||
            q.w_equation != NH_W_YAMAZAKI || !q.dry_zero)
            return fail(hd, NH_EINVAL,
                        "nh_adjoint_step: 2D non-hydrostatic steps of the h w_t = p form "
                        "without friction or breaking, q = 0 in dry cells, only");
        int rc = adjoint_alloc();
        if (rc != NH_OK) return rc;
        T* eb = static_cast<T*>(ebv);
        T* a1b = static_cast<T*>(a1bv);
        T* a2b = static_cast<T*>(a2bv);
        T* wb = static_cast<T*>(wbv);
        T* Hb = static_cast<T*>(Hbv);
        void* tp = const_cast<void*>(tape);
        const T dt = (T)dtd;
        // the forward's solver statistics and polling state are left as they were
        const long long it0 = hd->solver_iters;
        const int li0 = hd->last_iters[0], li1 = hd->last_iters[1];
        const double lr0 = hd->last_resid[0], lr1 = hd->last_resid[1];
        const int lsi = last_solve_iters, lcp = last_cheb_passes;
        const int fb0 = hd->fallbacks;
        const long long fbi0 = hd->fallback_iters;
        for (T* z : {aE0, aQ10, aQ20}) cudaMemsetAsync(z, 0, nc * sizeof(T), hd->s);
        cudaMemsetAsync(aW0, 0, nn * sizeof(T), hd->s);
        // stage 2: input U1, base U^n; its output is U^{n+1}
        rc = adjoint_stage(1, dt, tape_at(tp, 4), tape_at(tp, 5), tape_at(tp, 6), tape_at(tp, 7),
                           tape_at(tp, 3), tape_at(tp, 11), tape_at(tp, 12), tape_at(tp, 13),
                           tape_at(tp, 14), eb, a1b, a2b, wb, aE1, aQ11, aQ21, aW1, Hb);
        // stage 1: input U^n; its output is U1
        if (rc == NH_OK)
            rc = adjoint_stage(0, dt, tape_at(tp, 0), tape_at(tp, 1), tape_at(tp, 2),
                               tape_at(tp, 3), tape_at(tp, 3), tape_at(tp, 4), tape_at(tp, 8),
                               tape_at(tp, 9), tape_at(tp, 10), aE1, aQ11, aQ21, aW1, aE0, aQ10,
                               aQ20, aW0, Hb);
        adjoint_iters += hd->solver_iters - it0;
        hd->solver_iters = it0;
        hd->last_iters[0] = li0; hd->last_iters[1] = li1;
        hd->last_resid[0] = lr0; hd->last_resid[1] = lr1;
        last_solve_iters = lsi; last_cheb_passes = lcp;
        hd->fallbacks = fb0; hd->fallback_iters = fbi0;
        if (rc != NH_OK) return rc;
        cudaMemcpyAsync(eb, aE0, nc * sizeof(T), cudaMemcpyDeviceToDevice, hd->s);
        cudaMemcpyAsync(a1b, aQ10, nc * sizeof(T), cudaMemcpyDeviceToDevice, hd->s);
        cudaMemcpyAsync(a2b, aQ20, nc * sizeof(T), cudaMemcpyDeviceToDevice, hd->s);
        cudaMemcpyAsync(wb, aW0, nn * sizeof(T), cudaMemcpyDeviceToDevice, hd->s);
        cudaError_t e = cudaStreamSynchronize(hd->s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(hd, e, "nh_adjoint_step");
        return NH_OK;
    }
    long long adjoint_iters = 0;
    // choice between the two Chebyshev pass forms (shared-memory or register weights)
    static constexpr int kVT = 128;   // event slots: 64 timed passes
    int pass_variant = -1;
    int cheb_form() const override { return pass_variant; }
    int vt_next = 0, vt_used = 0, solves = 0;
    int vt_var[kVT / 2] = {}, vt_pass[kVT / 2] = {}, vt_solve[kVT / 2] = {}, vt_ok[kVT / 2] = {};
    cudaEvent_t vt_ev[kVT] = {};
    bool cyclic = false;   // the cyclic forms (nh_params.cheb_cyclic) are the candidates
    // candidates: the Jacobi forms 0 .. cheb_pass_forms() - 1, or the cyclic forms after them
    int cand0() const { return cyclic ? cheb_pass_forms<T>() : 0; }
    int ncand() const { return cyclic ? cheb_cyclic_forms<T>() : cheb_pass_forms<T>(); }
    int timed_variant() { return cand0() + vt_next++ % ncand(); }
    void choose_pass_variant()
    {
        const int v0 = cand0(), nv = ncand();
        double sum[16] = {};
        int cnt[16] = {};
        // the first pass of each form warms it up and is not counted
        for (int k = nv; k < vt_used / 2; ++k) {
            float ms = 0.f;
            if (vt_ok[k] && cudaEventElapsedTime(&ms, vt_ev[2 * k], vt_ev[2 * k + 1]) == cudaSuccess) {
                sum[vt_var[k]] += ms;
                cnt[vt_var[k]] += 1;
            }
        }
        cudaGetLastError();
        int best = v0;
        for (int v = v0 + 1; v < v0 + nv; ++v)
            if (cnt[v] && (!cnt[best] || sum[v] / cnt[v] < sum[best] / cnt[best])) best = v;
        pass_variant = best;
    }
    bool accept_stall = false;   // set during the adjoint's transposed solves

    // ---- FP64 solves by defect correction with FP32 inner solves (nh_params.refine_fp32):
    // round k takes r = b - M x in FP64 (x = 0 at first), scales it by an exact power of two
    // into FP32, solves M d = r with FP32 rows to a relative 1e-4 by the same
    // Chebyshev-scheduled passes (the 96x64 register form), and adds d to x in FP64, until
    // ||D^-1 r|| <= tol ||D^-1 b|| in FP64.  The FP64 rows decide convergence, so the
    // result meets the FP64 tolerance while the sweeps run at the FP32 rate.
    Bufs<float> B32{};
    Prm<float> P32{};
    SolveCtl* h_sctl32 = nullptr;
    bool refine = false;
    int last32 = 0;

    // FP32 passes on (B32.dp, B32.r) <-> (B32.v[0], B32.v[1]) until ctl32 is done; the
    // iterate ends in B32.v[0] when an odd number of passes did work.
    int run_inner32(int& sweeps, const float*& d)
    {
        const int K = cheb_sweeps_per_pass<float>();
        const unsigned polls = hd->prm.wait_polls > 0 ? (unsigned)hd->prm.wait_polls
                                                      : kDefaultWaitPolls;
        cudaMemsetAsync(B32.r, 0, nn * sizeof(float), hd->s);
        cudaMemsetAsync(B32.dp, 0, nn * sizeof(float), hd->s);
        int launched = 0;
        int batch = last32 > 2 ? last32 - 1 : 4;
        for (;;) {
            for (int k = 0; k < batch; ++k) {
                const bool odd = (launched++ & 1) != 0;
                float* xa = odd ? B32.v[0] : B32.dp;
                float* pa = odd ? B32.v[1] : B32.r;
                float* xb = odd ? B32.dp : B32.v[0];
                float* pb = odd ? B32.r : B32.v[1];
                int rc = 0;
                K_(NH_K_CHEB_PASS, [&] {
                    rc = launch_cheb_pass<float>(P32, hd->s, B32, xa, pa, xb, pb, B.partials,
                                                 hd->prm.cheb_cyclic ? cheb_pass_forms<float>() : 7,
                                                 polls, -1);
                });
                if (rc != 0) return fail(hd, NH_ECUDA, "Chebyshev pass launch failed");
            }
            cudaMemcpyAsync(h_sctl32, B32.sctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, hd->s);
            cudaError_t e = cudaStreamSynchronize(hd->s);
            if (e != cudaSuccess) return cuda_fail(hd, e, "inner pressure solve");
            if (h_sctl32->done) break;
            batch = 2;
        }
        if (h_sctl32->status == 6 || h_sctl32->status == 7)
            return fail(hd, NH_ETIMEOUT, "Chebyshev pass: a wait for staged copies ran out "
                                         "of polls (the solve was abandoned)");
        sweeps = h_sctl32->sweeps;
        last32 = sweeps / K;
        d = ((sweeps / K) & 1) ? B32.v[0] : B32.dp;
        return NH_OK;
    }

    int solve_refine(int stage)
    {
        if constexpr (sizeof(T) != 8) {
            return fail(hd, NH_EINVAL, "defect correction applies to FP64 handles");
        } else {
            const nh_params& q = hd->prm;
            const int K32 = cheb_sweeps_per_pass<float>();
            for (int k = 0; k < 5; ++k) {
                const T* src[5] = {B.cC, B.cW, B.cE, B.cS, B.cN};
                float* dst[5] = {B32.cC, B32.cW, B32.cE, B32.cS, B32.cN};
                launch_convert_from_double<float>(Ln, src[k], dst[k], nn);
            }
            cudaMemcpyAsync(h_sctl, B.sctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, hd->s);
            cudaError_t e = cudaStreamSynchronize(hd->s);
            if (e != cudaSuccess) return cuda_fail(hd, e, "pressure solve");
            if (h_sctl->status == 4) return fallback(stage, false);   // not diagonally dominant
            const double bdb = h_sctl->bdb, tol2 = q.tol * q.tol, tol_in = 1e-4;
            cudaMemsetAsync(B.dp, 0, nn * sizeof(T), hd->s);
            int total = 0;
            bool conv = false;
            double rr = 0.0;
            for (int round = 0; round < 16; ++round) {
                K_(NH_K_SOLVE_INIT, [&] {
                    launch_refine_resid(P, Ln, B, B.dp, B.r, B.partials, B.sctl, B32.sctl,
                                        tol_in * tol_in, q.max_iter, K32);
                });
                cudaMemcpyAsync(h_sctl, B.sctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, hd->s);
                if ((e = cudaStreamSynchronize(hd->s)) != cudaSuccess)
                    return cuda_fail(hd, e, "pressure solve");
                rr = h_sctl->rr;
                if (rr <= tol2 * bdb) { conv = true; break; }
                if (total >= q.max_iter) break;
                K_(NH_K_SOLVE_INIT, [&] { launch_refine_scale(Ln, B.r, B32.rhs, nn, B.sctl); });
                int sw = 0;
                const float* d = nullptr;
                const int rc = run_inner32(sw, d);
                if (rc != NH_OK) return rc;
                total += sw;
                K_(NH_K_SOLVE_INIT, [&] { launch_refine_add(Ln, B.dp, d, nn, B.sctl); });
            }
            hd->solver_iters += total;
            hd->last_iters[stage] = total;
            hd->last_resid[stage] = bdb > 0.0 ? std::sqrt(rr / bdb) : 0.0;
            if (conv) return NH_OK;
            // not there within the rounds or the cap: BiCGStab goes on from x in FP64
            return fallback(stage, true);
        }
    }

    int debug_hyp(double dtd, void* e, void* a, void* b, int where) override
    {
        if (dim == 2)
            launch_hyp2d<T>(P, Lc, B.eta, B.q1, B.q2, B.eta, B.q1, B.q2, B.H, T(0), T(1),
                            (T)dtd, B.etas, B.q1s, B.q2s, B.stctl);
        else
            launch_hyp1d<T>(P, Lc, B.eta, B.q1, B.eta, B.q1, B.H, T(0), T(1), (T)dtd, B.etas,
                            B.q1s, B.stctl);
        if (e) cudaMemcpyAsync(e, B.etas, nc * sizeof(T), kind_out(where), hd->s);
        if (a) cudaMemcpyAsync(a, B.q1s, nc * sizeof(T), kind_out(where), hd->s);
        if (b && dim == 2) cudaMemcpyAsync(b, B.q2s, nc * sizeof(T), kind_out(where), hd->s);
        cudaError_t er = cudaStreamSynchronize(hd->s);
        if (er != cudaSuccess) return cuda_fail(hd, er, "nh_debug_hyperbolic");
        return NH_OK;
    }

    int debug_stall_copies(int block) override
    {
        if (dim != 2 || hd->prm.solver != NH_SOLVER_CHEBYSHEV)
            return fail(hd, NH_EINVAL, "nh_debug_stall_copies: 2D Chebyshev handles only");
        stall_block = block;
        return NH_OK;
    }

    int debug_system(double dtd, const void* x, void* rhs, void* mx, int where) override
    {
        Bufs<T> D = B;  // the current state taken as U*
        D.etas = B.eta; D.q1s = B.q1; D.q2s = B.q2; D.q1k = B.q1; D.q2k = B.q2;
        const T de = (T)dtd;
        if (dim == 2)
            launch_asm2d<T>(P, Ln, D, B.w, B.w, T(0), T(1), de, 1, 0, 0.0, 1, 0, B.partials,
                            B.sctl);
        else
            launch_asm1d<T>(P, Ln, D, B.q1, B.q1, B.w, B.w, T(0), T(1), de);
        if (rhs) cudaMemcpyAsync(rhs, B.rhs, nn * sizeof(T), kind_out(where), hd->s);
        if (x && mx) {
            cudaMemcpyAsync(B.r, x, nn * sizeof(T), kind_in(where), hd->s);
            if (dim == 2) launch_matvec2d<T>(P, Ln, B, B.r, B.rh);
            else launch_tridiag_apply1d<T>(P, Ln, B, B.r, B.rh);
            cudaMemcpyAsync(mx, B.rh, nn * sizeof(T), kind_out(where), hd->s);
        }
        cudaError_t er = cudaStreamSynchronize(hd->s);
        if (er != cudaSuccess) return cuda_fail(hd, er, "nh_debug_system");
        return NH_OK;
    }
};

int check_grid(const nh_grid* g, const nh_params* p, std::string& why)
{
    if (!g || !p) { why = "null grid or params"; return 0; }
    if (g->dim != 1 && g->dim != 2) { why = "dim must be 1 or 2"; return 0; }
    if (g->nx < 2 || g->ny < 1 || (g->dim == 2 && g->ny < 2)) {
        why = "need nx >= 2 (and ny >= 2 in 2D, ny >= 1 rows in 1D)";
        return 0;
    }
    if (!(g->dx > 0.0) || (g->dim == 2 && !(g->dy > 0.0))) { why = "dx, dy must be > 0"; return 0; }
    const bool periodic = g->bc[0] == NH_BC_PERIODIC || g->bc[1] == NH_BC_PERIODIC;
    if (periodic && (g->dim != 1 || g->bc[0] != g->bc[1])) {
        why = "periodic boundaries: 1D channels, west and east both periodic";
        return 0;
    }
    for (int k = 0; k < 4; ++k)
        if (g->bc[k] != NH_BC_WALL && g->bc[k] != NH_BC_OUTFLOW && !(k < 2 && periodic)) {
            why = "bc must be WALL or OUTFLOW (or PERIODIC on both ends of a 1D channel)";
            return 0;
        }
    if ((double)g->nx * (double)g->ny > 2.0e9) { why = "grid too large"; return 0; }
    if (!(p->g > 0.0) || !(p->cfl > 0.0) || !(p->delta > 0.0) || p->hdry < 0.0 ||
        p->manning_n < 0.0 || !(p->tol > 0.0) || p->max_iter < 1) {
        why = "invalid physical or solver parameter";
        return 0;
    }
    if (p->precision != NH_FP64 && p->precision != NH_FP32) { why = "precision must be FP64 or FP32"; return 0; }
    if (p->solver != NH_SOLVER_BICGSTAB && p->solver != NH_SOLVER_CHEBYSHEV) { why = "unknown solver"; return 0; }
    if (p->eps_dp < 0.0) { why = "eps_dp must be >= 0"; return 0; }
    if (p->adjoint_frozen_limiter != 0 && p->adjoint_frozen_limiter != 1) {
        why = "adjoint_frozen_limiter must be 0 or 1";
        return 0;
    }
    const int nforms = p->precision == NH_FP32
                           ? cheb_pass_forms<float>() + cheb_cyclic_forms<float>()
                           : cheb_pass_forms<double>() + cheb_cyclic_forms<double>();
    if (p->cheb_form < -1 || p->cheb_form >= nforms) { why = "cheb_form out of range"; return 0; }
    if (p->cheb_cyclic != 0 && p->cheb_cyclic != 1) { why = "cheb_cyclic must be 0 or 1"; return 0; }
    if (p->w_equation != NH_W_YAMAZAKI && p->w_equation != NH_W_TRANSPORT) {
        why = "w_equation must be NH_W_YAMAZAKI or NH_W_TRANSPORT";
        return 0;
    }
    for (int k = 0; k < 4; ++k) {
        const double L = p->relax_width[k];
        const double len = k < 2 ? g->nx * g->dx : (double)g->ny * g->dy;
        if (!(L >= 0.0) || L > len) {
            why = "relax_width must be in [0, the domain's length]";
            return 0;
        }
        if (L > 0.0 && ((k < 2 && periodic) || (k >= 2 && g->dim == 1))) {
            why = "relaxation zones: not on periodic sides, west / east only in 1D";
            return 0;
        }
    }
    return 1;
}

}  // namespace

extern "C" {

int nh_default_params(nh_params* p)
{
    if (!p) return NH_EINVAL;
    p->g = 9.81; p->cfl = 0.9; p->delta = 1e-5; p->hdry = 1e-5; p->manning_n = 0.0;
    p->B1 = 0.15; p->B2 = 0.5; p->breaking = 0; p->nonhydrostatic = 1;
    p->solver = NH_SOLVER_CHEBYSHEV; p->tol = 1e-12; p->max_iter = 2000;
    p->precision = NH_FP64; p->fixed_dt = 0.0; p->eps_dp = 0.0;
    p->adjoint_frozen_limiter = 0;
    p->cheb_form = -1;
    p->w_equation = NH_W_YAMAZAKI;
    for (int k = 0; k < 4; ++k) p->relax_width[k] = 0.0;
    p->dry_zero = 1;
    p->wait_polls = 0;
    p->capture = 1;
    p->refine_fp32 = 0;
    p->fallback_block_nodes = 70000;
    p->cheb_cyclic = 1;
    return NH_OK;
}

int nh_cheb_forms(int precision)
{
    if (precision == NH_FP32) return cheb_pass_forms<float>();
    if (precision == NH_FP64) return cheb_pass_forms<double>();
    return NH_EINVAL;
}

int nh_cheb_cyclic_forms(int precision)
{
    if (precision == NH_FP32) return cheb_cyclic_forms<float>();
    if (precision == NH_FP64) return cheb_cyclic_forms<double>();
    return NH_EINVAL;
}

int nh_create(const nh_grid* grid, const double* H, const nh_params* params, void* stream,
              nh_handle** out)
{
    if (!out) return NH_EINVAL;
    *out = nullptr;
    std::string why;
    if (!H || !check_grid(grid, params, why)) return NH_EINVAL;
    nh_handle* h = new nh_handle();
    h->grid = *grid;
    h->prm = *params;
    h->s = (cudaStream_t)stream;
    int rc;
    if (params->precision == NH_FP32) {
        auto* im = new Impl<float>();
        h->impl.reset(im);
        rc = im->init(h, H);
    } else {
        auto* im = new Impl<double>();
        h->impl.reset(im);
        rc = im->init(h, H);
    }
    if (rc != NH_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return NH_OK;
}

int nh_set_state(nh_handle* h, const void* eta, const void* q1, const void* q2, const void* w,
                 const void* p, double t, int where)
{
    if (!h) return NH_EINVAL;
    if (where != NH_HOST && where != NH_DEVICE) return fail(h, NH_EINVAL, "bad where");
    int rc = h->impl->set_state(eta, q1, q2, w, p, where);
    if (rc == NH_OK) { h->t = t; h->steps = 0; h->nonfinite = 0; }
    return rc;
}

int nh_get_state(nh_handle* h, void* eta, void* q1, void* q2, void* w, void* p, double* t,
                 int where)
{
    if (!h) return NH_EINVAL;
    if (where != NH_HOST && where != NH_DEVICE) return fail(h, NH_EINVAL, "bad where");
    int rc = h->impl->get_state(eta, q1, q2, w, p, where);
    if (t) *t = h->t;
    return rc;
}

int nh_step(nh_handle* h, double dt, double* dt_taken)
{
    if (!h) return NH_EINVAL;
    if (!(dt > 0.0)) dt = h->prm.fixed_dt > 0.0 ? h->prm.fixed_dt : h->dt_next;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, NH_EINVAL, "no positive time step");
    int rc = h->impl->step(dt);
    if (rc == NH_OK || rc == NH_ENOCONV) {
        h->t += dt;
        h->dt_last = dt;
        ++h->steps;
    }
    if (dt_taken) *dt_taken = dt;
    return rc;
}

int nh_run(nh_handle* h, double t_end, long long max_steps, long long* steps_taken)
{
    if (!h) return NH_EINVAL;
    long long s = 0;
    int rc = NH_OK;
    while (s < max_steps) {
        if (t_end > 0.0 && h->t >= t_end) break;
        double dt = h->prm.fixed_dt > 0.0 ? h->prm.fixed_dt : h->dt_next;
        if (!(dt > 0.0)) break;
        if (t_end > 0.0 && h->t + dt > t_end) dt = t_end - h->t;
        rc = nh_step(h, dt, nullptr);
        if (rc != NH_OK) break;
        ++s;
    }
    if (steps_taken) *steps_taken = s;
    return rc;
}

int nh_gauges(nh_handle* h, const int* cells, int n, void* out)
{
    if (!h || n < 0 || (n > 0 && (!cells || !out))) return NH_EINVAL;
    if (n == 0) return NH_OK;
    return h->impl->gauges(cells, n, out);
}

int nh_stats(nh_handle* h, nh_stats_t* out)
{
    if (!h || !out) return NH_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->t = h->t;
    out->dt = h->dt_last;
    out->dt_next = h->dt_next;
    out->steps = h->steps;
    out->solver_iters = h->solver_iters;
    out->last_iters[0] = h->last_iters[0];
    out->last_iters[1] = h->last_iters[1];
    out->last_resid[0] = h->last_resid[0];
    out->last_resid[1] = h->last_resid[1];
    out->nonfinite = h->nonfinite;
    out->fallbacks = h->fallbacks;
    out->fallback_iters = h->fallback_iters;
    out->cheb_form =
        h->prm.solver == NH_SOLVER_CHEBYSHEV && h->grid.dim == 2 ? h->impl->cheb_form() : -1;
    return h->impl->mass(&out->mass);
}

const char* nh_last_error(const nh_handle* h)
{
    return h ? h->err.c_str() : "null handle";
}

void nh_destroy(nh_handle* h)
{
    if (!h) return;
    if (h->s) cudaStreamSynchronize(h->s);
    else cudaDeviceSynchronize();
    delete h;
}

int nh_profile_enable(nh_handle* h, int on)
{
    if (!h) return NH_EINVAL;
    return h->impl->profile_enable(on);
}

int nh_profile_read(nh_handle* h, nh_profile_t* out)
{
    if (!h || !out) return NH_EINVAL;
    return h->impl->profile_read(out);
}

int nh_set_relax_target(nh_handle* h, const void* eta, const void* q1, const void* q2,
                        const void* w, const void* p, int where)
{
    if (!h) return NH_EINVAL;
    if (where != NH_HOST && where != NH_DEVICE) return fail(h, NH_EINVAL, "bad where");
    return h->impl->set_relax_target(eta, q1, q2, w, p, where);
}

int nh_debug_hyperbolic(nh_handle* h, double dt, void* eta_out, void* q1_out, void* q2_out,
                        int where)
{
    if (!h || !(dt > 0.0)) return NH_EINVAL;
    return h->impl->debug_hyp(dt, eta_out, q1_out, q2_out, where);
}

size_t nh_tape_bytes(nh_handle* h)
{
    return h ? h->impl->tape_bytes() : 0;
}

int nh_step_taped(nh_handle* h, double dt, void* tape, double* dt_taken)
{
    if (!h || !tape) return NH_EINVAL;
    if (h->grid.dim != 2) return fail(h, NH_EINVAL, "nh_step_taped: 2D only");
    if (h->prm.w_equation != NH_W_YAMAZAKI)
        return fail(h, NH_EINVAL, "nh_step_taped: the adjoint covers the h w_t = p form only");
    if (!h->prm.dry_zero)
        return fail(h, NH_EINVAL, "nh_step_taped: the adjoint covers q = 0 in dry cells "
                                  "(dry_zero = 1) only");
    for (int k = 0; k < 4; ++k)
        if (h->prm.relax_width[k] > 0.0)
            return fail(h, NH_EINVAL, "nh_step_taped: the adjoint covers steps without "
                                      "relaxation zones only");
    const double d = dt > 0.0 ? dt : h->dt_next;
    if (!(d > 0.0)) return fail(h, NH_EINVAL, "no positive time step");
    int rc = h->impl->step_taped(d, tape);
    if (rc == NH_OK || rc == NH_ENOCONV) {
        h->t += d;
        h->dt_last = d;
        h->steps += 1;
        if (dt_taken) *dt_taken = d;
    }
    return rc;
}

int nh_adjoint_step(nh_handle* h, double dt, const void* tape, void* eta_bar, void* q1_bar,
                    void* q2_bar, void* w_bar, void* H_bar)
{
    if (!h || !tape || !eta_bar || !q1_bar || !q2_bar || !w_bar || !H_bar || !(dt > 0.0))
        return NH_EINVAL;
    return h->impl->adjoint_step(dt, tape, eta_bar, q1_bar, q2_bar, w_bar, H_bar);
}

int nh_debug_stall_copies(nh_handle* h, int block)
{
    if (!h || block < 0) return NH_EINVAL;
    return h->impl->debug_stall_copies(block);
}

int nh_debug_system(nh_handle* h, double dt, const void* x, void* rhs_out, void* mx_out,
                    int where)
{
    if (!h || !(dt > 0.0)) return NH_EINVAL;
    return h->impl->debug_system(dt, x, rhs_out, mx_out, where);
}

}  // extern "C"
