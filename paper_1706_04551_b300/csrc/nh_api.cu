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
    virtual int lambda(double* lam) = 0;
    virtual int mass(double* m) = 0;
    virtual int debug_hyp(double dt, void* e, void* a, void* b, int where) = 0;
    virtual int debug_system(double dt, const void* x, void* rhs, void* mx, int where) = 0;
    virtual int profile_enable(int on) = 0;
    virtual int profile_read(nh_profile_t* out) = 0;
};

// Event pairs around kernel launches, accumulated per kernel class.
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<int> cls;
    size_t used = 0;
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
    void flush()
    {
        if (used == 0) return;
        cudaEventSynchronize(pool[used - 1]);
        for (size_t k = 0; k < cls.size(); ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, pool[2 * k], pool[2 * k + 1]);
            ms[cls[k]] += t;
            launches[cls[k]] += 1;
        }
        used = 0;
        cls.clear();
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
    Bufs<T> B;
    std::vector<void*> allocs;
    Prof prof;
    SolveCtl* h_sctl = nullptr;   // pinned mirrors of the device control blocks
    StepCtl* h_stctl = nullptr;
    int last_solve_iters = 0;
    int last_cheb_passes = 0;

    ~Impl() override
    {
        for (void* p : allocs) cudaFree(p);
        if (h_sctl) cudaFreeHost(h_sctl);
        if (h_stctl) cudaFreeHost(h_stctl);
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
        P.B1 = (T)q.B1; P.breaking = q.breaking;
        nc = (size_t)g.nx * g.ny;
        nn = dim == 2 ? (size_t)(g.nx + 1) * (g.ny + 1) : (size_t)(g.nx + 1) * g.ny;
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 148;
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
#undef A
        cudaError_t e;
        if ((e = cudaMallocHost(&h_sctl, sizeof(SolveCtl))) != cudaSuccess) return cuda_fail(hd, e, "cudaMallocHost");
        if ((e = cudaMallocHost(&h_stctl, sizeof(StepCtl))) != cudaSuccess) return cuda_fail(hd, e, "cudaMallocHost");
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
        cudaEventRecord(prof.next(), hd->s);
        f();
        cudaEventRecord(prof.next(), hd->s);
        prof.cls.push_back(cls);
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
        double lam = 0.0;
        int rc = lambda(&lam);
        if (rc != NH_OK) return rc;
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

    int lambda(double* lam) override
    {
        launch_lambda<T>(P, Lc, B.eta, B.q1, B.q2, B.H, dim, B.partials, B.stctl);
        cudaMemcpyAsync(h_stctl, B.stctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, hd->s);
        cudaError_t e = cudaStreamSynchronize(hd->s);
        if (e != cudaSuccess) return cuda_fail(hd, e, "lambda");
        *lam = h_stctl->lam;
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
    int solve_cheb(int stage)
    {
        const int K = cheb_sweeps_per_pass<T>();
        cudaMemsetAsync(B.r, 0, nn * sizeof(T), hd->s);
        cudaMemsetAsync(B.dp, 0, nn * sizeof(T), hd->s);
        int batch = last_cheb_passes > 2 ? last_cheb_passes - 1 : 4;
        double best = 1e300;
        int stale = 0;
        for (;;) {
            for (int k = 0; k < batch; ++k) {
                int rc = 0;
                K_(NH_K_CHEB_PASS, [&] { rc = launch_cheb_pass<T>(P, hd->s, B, B.r, B.partials); });
                if (rc != 0) return fail(hd, NH_ECUDA, "Chebyshev pass launch failed");
            }
            cudaMemcpyAsync(h_sctl, B.sctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, hd->s);
            cudaError_t e = cudaStreamSynchronize(hd->s);
            if (e != cudaSuccess) return cuda_fail(hd, e, "pressure solve");
            if (h_sctl->status == 4) return fallback(stage, false);   // not diagonally dominant
            if (h_sctl->done) break;
            // stagnation (rounding floor of the precision, or a spectrum the Gershgorin
            // interval does not describe): continue with BiCGStab from the current dp
            if (h_sctl->rr < 0.81 * best) { best = h_sctl->rr; stale = 0; }
            else if (++stale >= 4) {
                const int done_sweeps = h_sctl->sweeps;
                hd->solver_iters += done_sweeps;
                last_cheb_passes = done_sweeps / K;
                return fallback(stage, true);
            }
            batch = 2;
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
        K_(NH_K_HYPERBOLIC, [&] {
            launch_hyp2d<T>(P, Lc, ein, ain, bin, B.eta, B.q1, B.q2, B.H, a, b, dt, B.etas,
                            B.q1s, B.q2s, B.stctl);
        });
        if (q.breaking)
            K_(NH_K_BREAKING, [&] {
                launch_break2d<T>(P, Lc, B.etas, B.q1s, B.q2s, B.H, de, B.q1k, B.q2k);
            });
        K_(NH_K_ASSEMBLY, [&] {
            launch_asm2d<T>(P, Ln, B, win, B.w, a, b, de, q.nonhydrostatic ? 1 : 0,
                            q.nonhydrostatic ? 1 : 0, q.tol * q.tol, q.max_iter,
                            q.solver == NH_SOLVER_CHEBYSHEV ? cheb_sweeps_per_pass<T>() : 0,
                            B.partials, B.sctl);
        });
        int rc = NH_OK;
        if (q.nonhydrostatic) rc = q.solver == NH_SOLVER_CHEBYSHEV ? solve_cheb(s) : solve2d(s, false);
        K_(NH_K_CORRECTION, [&] {
            launch_corr2d<T>(P, Ln, B, B.q1k, B.q2k, de, q.nonhydrostatic ? 1 : 0, eo, ao, bo,
                             wo, s == 1 ? 1 : 0, B.partials, B.stctl);
        });
        std::swap(B.p, B.palt);
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
        K_(NH_K_HYPERBOLIC, [&] {
            launch_hyp1d<T>(P, Lc, ein, ain, B.eta, B.q1, B.H, a, b, dt, B.etas, B.q1s, B.stctl);
        });
        if (q.breaking)
            K_(NH_K_BREAKING, [&] { launch_break1d<T>(P, Lc, B.etas, B.q1s, B.H, de, B.q1k); });
        K_(NH_K_ASSEMBLY, [&] { launch_asm1d<T>(P, Ln, B, B.q1s, B.q1k, win, B.w, a, b, de); });
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
        const T dt = (T)dtd;
        cudaMemsetAsync(&B.stctl->clamped, 0, sizeof(int), hd->s);
        int rc1 = dim == 2 ? stage2d(0, dt) : stage1d(0, dt);
        if (rc1 != NH_OK && rc1 != NH_ENOCONV) return rc1;
        int rc2 = dim == 2 ? stage2d(1, dt) : stage1d(1, dt);
        if (rc2 != NH_OK && rc2 != NH_ENOCONV) return rc2;
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
    for (int k = 0; k < 4; ++k)
        if (g->bc[k] != NH_BC_WALL && g->bc[k] != NH_BC_OUTFLOW) { why = "bc must be WALL or OUTFLOW"; return 0; }
    if ((double)g->nx * (double)g->ny > 2.0e9) { why = "grid too large"; return 0; }
    if (!(p->g > 0.0) || !(p->cfl > 0.0) || !(p->delta > 0.0) || p->hdry < 0.0 ||
        p->manning_n < 0.0 || !(p->tol > 0.0) || p->max_iter < 1) {
        why = "invalid physical or solver parameter";
        return 0;
    }
    if (p->precision != NH_FP64 && p->precision != NH_FP32) { why = "precision must be FP64 or FP32"; return 0; }
    if (p->solver != NH_SOLVER_BICGSTAB && p->solver != NH_SOLVER_CHEBYSHEV) { why = "unknown solver"; return 0; }
    if (p->eps_dp < 0.0) { why = "eps_dp must be >= 0"; return 0; }
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
    return NH_OK;
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

int nh_debug_hyperbolic(nh_handle* h, double dt, void* eta_out, void* q1_out, void* q2_out,
                        int where)
{
    if (!h || !(dt > 0.0)) return NH_EINVAL;
    return h->impl->debug_hyp(dt, eta_out, q1_out, q2_out, where);
}

int nh_debug_system(nh_handle* h, double dt, const void* x, void* rhs_out, void* mx_out,
                    int where)
{
    if (!h || !(dt > 0.0)) return NH_EINVAL;
    return h->impl->debug_system(dt, x, rhs_out, mx_out, where);
}

}  // extern "C"
