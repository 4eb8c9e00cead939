// Full-lattice solves through the even-odd Schur system.
//
// D x = eta (FULL_DIRAC):
//   eta~_e = M^-1 (eta_e - H_eo M^-1 eta_o);  S x_e = eta~_e solved as S^dag S x_e = S^dag eta~_e;
//   x_o = M^-1 (eta_o - H_oe x_e).
// D^dag D x = b (FULL_NORMAL) as y = D^-dag b, then x = D^-1 y.  With
// M^dag - H_oe^dag M^-dag H_eo^dag = S^dag M^dag:
//   z_e = b_e - H_oe^dag M^-dag b_o;  v = (S^dag S)^-1 z_e;  y_e = M^-dag S v;
//   y_o = M^-dag (b_o - H_eo^dag y_e).
// Every solve of S^dag S uses the batched CG.  The composed solves amplify the inner
// tolerance, so the FP64 residual of the full system is recomputed on the full lattice and
// the pipeline is re-run on it (iterative refinement) until it meets the tolerance.
#include <chrono>
#include <cmath>

#include "batch_cg.h"
#include "engine.h"

namespace odwf {

namespace {

// one S^dag S solve: B64 slot 0 of `bc` must hold the right-hand side
int run_cg(BatchCG& bc, double mqv, cudaStream_t st, int every, int* iters, int* nrel, int* status) {
    int rc = 0;
    bc.mq[0] = mqv;
    if ((rc = bc.admit_internal(0, st))) return rc;
    while (true) {
        if ((rc = bc.resume(st, true))) return rc;
        if ((rc = bc.run_iterations(every, st))) return rc;
        if ((rc = bc.poll(st))) return rc;
        if ((rc = bc.service(st))) return rc;
        if (!bc.any_running()) break;
    }
    double tr = 0;
    if ((rc = bc.finalize(0, nullptr, st, &tr))) return rc;
    *iters += bc.st_host[0].iter;
    *nrel += bc.n_reliable[0];
    *status = bc.st_host[0].status;
    return ODWF_OK;
}

}  // namespace

int Engine::solve_full(void* x, const void* b, const odwf_solve_params* prm, odwf_solve_stats* stats,
                       cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const int system = prm->system;
    if (system != ODWF_SYS_FULL_DIRAC && system != ODWF_SYS_FULL_NORMAL)
        return fail(ODWF_EINVAL, "solve: unknown system");
    const double mqv = std::isfinite(prm->mq) ? prm->mq : mq;
    int rc = 0;
    // r of this solve for the FP64 operator kernels
    double* rd = (double*)get_ws("r_solve", sizeof(double), &rc);
    if (rc) return rc;
    const double rv = mqv / (2.0 * m0);
    ODWF_CK(cudaMemcpy(rd, &rv, sizeof(double), cudaMemcpyHostToDevice));

    const size_t eb = ext_bytes(ODWF_MODE_FULL);
    const double2* db = nullptr;
    if (is_device_ptr(b)) {
        db = (const double2*)b;
    } else {
        void* d = get_ws("ext.in", eb, &rc);
        if (rc) return rc;
        ODWF_CK(cudaMemcpyAsync(d, b, eb, cudaMemcpyHostToDevice, st));
        db = (const double2*)d;
    }
    const bool x_dev = is_device_ptr(x);
    double2* dx = x_dev ? (double2*)x : (double2*)get_ws("ext.out", eb, &rc);
    if (rc) return rc;

    HalfField Be, Bo, Re, Ro, Ye, Yo, Xe, Xo, Ee, Eo, W, U, Ze, Zo;
    const char* names[] = {"fs.Be", "fs.Bo", "fs.Re", "fs.Ro", "fs.Ye", "fs.Yo", "fs.Xe",
                           "fs.Xo", "fs.Ee", "fs.Eo", "fs.W", "fs.U", "fs.Ze", "fs.Zo"};
    HalfField* fields[] = {&Be, &Bo, &Re, &Ro, &Ye, &Yo, &Xe, &Xo, &Ee, &Eo, &W, &U, &Ze, &Zo};
    for (int k = 0; k < 14; ++k)
        if ((rc = alloc_half(names[k], Sp::F64, 1, fields[k]))) return rc;
    ODWF_CK(launch_pack(Sp::F64, db, Be.ref_sys(0), g, 0, ns, 0, st));
    ODWF_CK(launch_pack(Sp::F64, db, Bo.ref_sys(0), g, 1, ns, 0, st));

    BatchCG bc;
    // the pipeline reads and writes the CG's solution and right-hand side with the FP64 kernels
    odwf_solve_params prm64 = *prm;
    prm64.update_arith = ODWF_UPDATES_F64;
    if ((rc = bc.init(this, 1, prm64, st))) return rc;
    const int every = prm->check_every > 0 ? prm->check_every : 8;
    int iters = 0, nrel = 0, status = kDone;
    const size_t n5 = sites5();
    auto copy = [&](const HalfField& a, const HalfField& b) {
        return launch_vec(Sp::F64, Sp::F64, a.ref_sys(0), b.ref_sys(0), n5, ns, 0, 0.0, nullptr, 0, 0, nullptr,
                          nullptr, 0, 1, st);
    };
    auto axpy = [&](double c, const HalfField& a, const HalfField& b) {  // b += c a
        return launch_vec(Sp::F64, Sp::F64, a.ref_sys(0), b.ref_sys(0), n5, ns, 4, c, nullptr, 0, 0, nullptr,
                          nullptr, 0, 1, st);
    };
    auto norm2 = [&](const HalfField& a, double* out) -> int {
        ODWF_CK(launch_vec(Sp::F64, Sp::F64, a.ref_sys(0), a.ref_sys(0), n5, ns, 3, 0.0, bc.st, 0, 0, bc.partials,
                           bc.counters, 0, 1, st));
        ODWF_CK(cudaMemcpyAsync(out, &bc.st[0].sum, sizeof(double), cudaMemcpyDeviceToHost, st));
        ODWF_CK(cudaStreamSynchronize(st));
        return ODWF_OK;
    };

    // One pass of the Schur pipeline: E = A^-1 R (approximately, to the CG tolerance).
    auto solve_once = [&]() -> int {
        // Y = right-hand side of the D solve (R itself for FULL_DIRAC, D^-dag R for FULL_NORMAL)
        if (system == ODWF_SYS_FULL_NORMAL) {
            // W = M^-dag r_o;  bc.B64 = z_e = r_e - H_oe^dag W
            ODWF_CK(launch_m5_f64(Ro.ref_sys(0), W.ref_sys(0), vh(), ns, rd, 0, 1, 3, cf64, st));
            auto P = hop_params<double>(0, rd);
            P.in = W.ref_sys(0);
            P.z = Re.ref_sys(0);
            P.out = bc.B64.ref_sys(0);
            ODWF_CK(launch_hop_f64(P, Epi::D_ZMINUS, 1, st));
            int s1 = 0, r1 = run_cg(bc, mqv, st, every, &iters, &nrel, &s1);
            if (r1) return r1;
            if (s1 != kDone) status = s1;
            // y_e = M^-dag S v  (v in bc.X64)
            if ((r1 = apply_schur64(bc.X64, U, false, rd, st))) return r1;
            ODWF_CK(launch_m5_f64(U.ref_sys(0), Ye.ref_sys(0), vh(), ns, rd, 0, 1, 3, cf64, st));
            // y_o = M^-dag (r_o - H_eo^dag y_e)
            P = hop_params<double>(1, rd);
            P.in = Ye.ref_sys(0);
            P.z = Ro.ref_sys(0);
            P.out = Yo.ref_sys(0);
            ODWF_CK(launch_hop_f64(P, Epi::D_ZMINUS_POSTMINVDAG, 1, st));
        } else {
            ODWF_CK(copy(Re, Ye));
            ODWF_CK(copy(Ro, Yo));
        }
        // D e = y:  W = M^-1 y_o;  U = eta~_e = M^-1 (y_e - H_eo W);  bc.B64 = S^dag U
        ODWF_CK(launch_m5_f64(Yo.ref_sys(0), W.ref_sys(0), vh(), ns, rd, 0, 1, 2, cf64, st));
        auto P = hop_params<double>(0, rd);
        P.in = W.ref_sys(0);
        P.z = Ye.ref_sys(0);
        P.out = U.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::ZMINUS_POSTMINV, 1, st));
        int r2 = apply_schur64(U, bc.B64, true, rd, st);
        if (r2) return r2;
        int s2 = 0;
        if ((r2 = run_cg(bc, mqv, st, every, &iters, &nrel, &s2))) return r2;
        if (s2 != kDone) status = s2;
        ODWF_CK(copy(bc.X64, Ee));
        // e_o = M^-1 (y_o - H_oe e_e)
        P = hop_params<double>(1, rd);
        P.in = Ee.ref_sys(0);
        P.z = Yo.ref_sys(0);
        P.out = Eo.ref_sys(0);
        ODWF_CK(launch_hop_f64(P, Epi::ZMINUS_POSTMINV, 1, st));
        return ODWF_OK;
    };

    // Outer FP64 iterative refinement: the composed Schur solves amplify the inner tolerance,
    // so the full-system residual is recomputed and the solve repeated on it until it meets tol.
    double bb = 0, be = 0, bo = 0;
    if ((rc = norm2(Be, &be)) || (rc = norm2(Bo, &bo))) return rc;
    bb = be + bo;
    ODWF_CK(copy(Be, Re));
    ODWF_CK(copy(Bo, Ro));
    ODWF_CK(launch_vec(Sp::F64, Sp::F64, Xe.ref_sys(0), Xe.ref_sys(0), n5, ns, 5, 0.0, nullptr, 0, 0, nullptr,
                       nullptr, 0, 1, st));
    ODWF_CK(launch_vec(Sp::F64, Sp::F64, Xo.ref_sys(0), Xo.ref_sys(0), n5, ns, 5, 0.0, nullptr, 0, 0, nullptr,
                       nullptr, 0, 1, st));
    double tr = 0.0;
    const int max_rounds = 6;
    for (int round = 0; round < max_rounds && bb > 0; ++round) {
        if ((rc = solve_once())) return rc;
        ODWF_CK(axpy(1.0, Ee, Xe));
        ODWF_CK(axpy(1.0, Eo, Xo));
        // R = B - A X in FP64, A = D (FULL_DIRAC) or D^dag D (FULL_NORMAL)
        if ((rc = apply_full64(Xe, Xo, Ze, Zo, false, rd, st))) return rc;
        if (system == ODWF_SYS_FULL_NORMAL) {
            if ((rc = apply_full64(Ze, Zo, W, U, true, rd, st))) return rc;
        } else {
            ODWF_CK(copy(Ze, W));
            ODWF_CK(copy(Zo, U));
        }
        ODWF_CK(copy(Be, Re));
        ODWF_CK(copy(Bo, Ro));
        ODWF_CK(axpy(-1.0, W, Re));
        ODWF_CK(axpy(-1.0, U, Ro));
        double re = 0, ro = 0;
        if ((rc = norm2(Re, &re)) || (rc = norm2(Ro, &ro))) return rc;
        tr = std::sqrt((re + ro) / bb);
        if (tr <= prm->tol || status == kBreakdown) break;
        if (iters >= prm->max_iter) break;
    }
    if (bb > 0 && tr > prm->tol && status == kDone) status = kMaxIter;
    ODWF_CK(launch_unpack(Sp::F64, Xe.ref_sys(0), dx, g, 0, ns, 0, st));
    ODWF_CK(launch_unpack(Sp::F64, Xo.ref_sys(0), dx, g, 1, ns, 0, st));
    if (!x_dev) {
        ODWF_CK(cudaMemcpyAsync(x, dx, eb, cudaMemcpyDeviceToHost, st));
    }
    ODWF_CK(cudaStreamSynchronize(st));
    int code = ODWF_OK;
    if (status == kBreakdown) code = ODWF_EBREAKDOWN;
    else if (status != kDone) code = ODWF_ENOCONV;
    if (stats) {
        stats->iters = iters;
        stats->n_reliable = nrel;
        stats->true_resid = tr;
        stats->status = code;
        stats->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (code == ODWF_ENOCONV) set_error("solve: max_iter reached before the tolerance");
    if (code == ODWF_EBREAKDOWN) set_error("solve: CG breakdown");
    return code;
}

}  // namespace odwf
