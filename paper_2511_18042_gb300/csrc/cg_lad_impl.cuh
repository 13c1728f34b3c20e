// LAD and hybrid stage orchestration (included by cg_api.cu after the
// C-GBR helpers).  Algorithm 1 (LAD: node fluxes, viscous/LAD terms, residual,
// RK update, filter on the last stage), Algorithm 3 (hybrid: the whole stage
// by GBR if a troubled cell exists, else LAD) and its per-interface variant.

static int lad_alloc(cg_solver* s) {
  int sch = s->p.scheme;
  if (sch != CG_LAD_E4 && sch != CG_LAD_C6 && sch != CG_HYBRID && !s->p.viscous) return CG_OK;
  LadBuffers& L = s->lad;
  int nd = s->nd, nv = s->nv, nf = nd + 3;
  L.fbx = make_box(s, 8, -1, 8);
  L.b3 = make_box(s, 3, -1, 3);
  L.tbox = make_box(s, 1, -1, 1);
  L.ubx = make_box(s, 2, -1, 2);
  size_t fmax = 0;
  for (int d = 0; d < nd; ++d) {
    L.fbox[d] = make_box(s, 0, d, 2);
    Box hb = make_box(s, 0, d, 0);
    hb.off[d] = 1;
    hb.ext[d] = s->dg.n[d] + 1;
    L.hbox[d] = hb;
    s->hBox[d] = hb;
    fmax = std::max(fmax, (size_t)L.fbox[d].size());
  }
  int rc;
  if ((rc = dalloc(&L.fb, (size_t)nf * L.fbx.size())) || (rc = dalloc(&L.gr, (size_t)nf * nd * L.b3.size())) ||
      (rc = dalloc(&L.dv, (size_t)L.b3.size())) || (rc = dalloc(&L.bt[0], (size_t)s->N)) ||
      (rc = dalloc(&L.bt[1], (size_t)s->N)) || (rc = dalloc(&L.kp[0], (size_t)s->N)) ||
      (rc = dalloc(&L.kp[1], (size_t)s->N)) || (rc = dalloc(&L.Fn, (size_t)nv * fmax * nd)))
    return rc;
  L.fstride = (size_t)nv * fmax;
  if (s->p.viscous) {
    L.vbx = make_box(s, 2, -1, 2);
    if ((rc = dalloc(&L.vco, (size_t)3 * L.vbx.size()))) return rc;
  }
  if (sch == CG_LAD_C6) {
    size_t dmax = 0, fl = 0;
    long long grad_cols = 0, flux_cols = 0;
    for (int d = 0; d < nd; ++d) {
      int n = s->dg.n[d];
      L.dfLB[d] = make_lines(s, d, -6, n + 12, 3);
      L.DLB[d] = make_lines(s, d, 0, n, 0);
      L.filtLB[d] = make_lines(s, d, -1, n + 2, 0);
      grad_cols += L.dfLB[d].nl * nf;
      flux_cols += L.DLB[d].nl * nv;
    }
    for (int d = 0; d < nd; ++d) {
      bool cyc = s->grid->bc[d][0] == CG_BC_PERIODIC;
      int n = s->dg.n[d];
      if (cyc && n < 3) return fail(CG_ERR_INVALID_ARG, "periodic compact lines need n >= 3");
      if ((rc = dalloc(&L.df[d], (size_t)nf * L.dfLB[d].m * L.dfLB[d].nl))) return rc;
      dmax = std::max(dmax, (size_t)nv * (size_t)L.DLB[d].m * (size_t)L.DLB[d].nl);
      fl = std::max(fl, (size_t)nv * (size_t)L.filtLB[d].m * (size_t)L.filtLB[d].nl);
      if ((rc = upload_line(s->c6grad[d], cyc ? n : n + 12, 1.0 / 3.0, cyc, -6, grad_cols))) return rc;
      // all directions' flux lines are solved in one launch: partitions for their total
      if ((rc = upload_line(s->c6flux[d], n, 1.0 / 3.0, cyc, 0, flux_cols))) return rc;
      if ((rc = upload_line(s->filt[d], cyc ? n : n + 2, s->p.alpha_f, cyc, -1, L.filtLB[d].nl * nv))) return rc;
    }
    // LAD-C6: node fluxes and derivatives of every direction held at once (one
    // launch solves all directions' flux lines)
    if ((rc = dalloc(&L.D, dmax * nd)) || (rc = dalloc(&L.lines, fl))) return rc;
    L.dstride = dmax;
  }
  if (sch == CG_HYBRID) {
    if ((rc = dalloc(&L.tr, (size_t)L.tbox.size()))) return rc;
    // interface fluxes in the arithmetic type of the LAD pass and the sweep
    // (FP32 in the mixed form, stored in half as many doubles)
    for (int d = 0; d < nd; ++d) {
      size_t cnt = (size_t)nv * L.hbox[d].size();
      if (s->p.precision == CG_MIXED) cnt = (cnt + 1) / 2;
      if ((rc = dalloc(&s->hflux[d], cnt))) return rc;
    }
  }
  return CG_OK;
}

static void lad_free(LadBuffers& L) {
  double* bufs[] = {L.fb, L.gr, L.dv, L.bt[0], L.bt[1], L.kp[0], L.kp[1], L.Fn, L.D, L.df[0], L.df[1], L.df[2], L.lines,
                    L.vco};
  for (double* b : bufs)
    if (b) cudaFree(b);
  if (L.tr) cudaFree(L.tr);
}

// beta*, kappa* (filtered, interior) of the primitives in s->W; result in
// bt[0], kp[0].  dkind: 2 = E4, 3 = C6.
template <int ND, typename T = double>
static int lad_coeffs_run(cg_solver* s, int dkind, cudaStream_t st, const int* guard, int want) {
  LadBuffers& L = s->lad;
  bool c6 = dkind == 3;
  T* fb = reinterpret_cast<T*>(L.fb);
  T* gr = reinterpret_cast<T*>(L.gr);
  T* dv = reinterpret_cast<T*>(L.dv);
  T* bt[2] = {reinterpret_cast<T*>(L.bt[0]), reinterpret_cast<T*>(L.bt[1])};
  T* kp[2] = {reinterpret_cast<T*>(L.kp[0]), reinterpret_cast<T*>(L.kp[1])};
  k_lad_fieldbuf<ND, T><<<grid_blocks(L.fbx.size(), 256), 256, 0, st>>>(s->dg, reinterpret_cast<const T*>(s->W), fb, L.fbx);
  s->launches++;
  T* df[3] = {reinterpret_cast<T*>(L.df[0]), reinterpret_cast<T*>(L.df[1]), reinterpret_cast<T*>(L.df[2])};
  if (c6) {
    LineJob<T> jobs[3];
    for (int l = 0; l < ND; ++l) jobs[l] = LineJob<T>{&s->c6grad[l], df[l], L.dfLB[l].nl, ND + 3};
    const bool fused = rhs_in_solver(jobs, ND);  // the solver forms the right-hand sides
    for (int l = 0; l < ND; ++l) {
      const LineBuf& lb = L.dfLB[l];
      if (fused) {
        jobs[l].src = C6Src<T>{fb, L.fbx, L.fbx.size(), lb};
      } else {
        launch_rhs_c6<ND, T>(fb, L.fbx, ND + 3, lb, df[l], st);
        s->launches++;
      }
    }
    launch_lines(jobs, ND, st);
    s->launches++;
  }
  int gb = grid_blocks(L.b3.size(), 128);
  const dim3 xt_grid((unsigned)((L.b3.ext[0] + LGT_X - 1) / LGT_X), (unsigned)((L.b3.ext[1] + LGT_Y - 1) / LGT_Y),
                     ND == 3 ? (unsigned)L.b3.ext[2] : 1u);
  const bool xt = ND >= 2 && c6;  // C6 in 2D/3D: the x lines through the tiled read
  if (s->dg.curv) {
    if (xt) {
      if constexpr (ND >= 2)
        k_lad_grad_xt<ND, false, T><<<xt_grid, dim3(LGT_X, LGT_Y), 0, st>>>(s->dg, df[0], df[1], df[2], L.dfLB[0],
                                                                           L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
    }
    else if (c6) k_lad_grad<ND, false, true, T><<<gb, 128, 0, st>>>(s->dg, fb, L.fbx, df[0], df[1], df[2], L.dfLB[0], L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
    else k_lad_grad<ND, false, false, T><<<gb, 128, 0, st>>>(s->dg, fb, L.fbx, df[0], df[1], df[2], L.dfLB[0], L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
    k_lad_coef<ND, false, T><<<grid_blocks(s->N, 128), 128, 0, st>>>(s->dg, reinterpret_cast<const T*>(s->W), fb, L.fbx, gr, dv, L.b3, s->p.c_beta,
                                                                     s->p.c_kappa, bt[0], kp[0], guard, want);
  } else {
    if (xt) {
      if constexpr (ND >= 2)
        k_lad_grad_xt<ND, true, T><<<xt_grid, dim3(LGT_X, LGT_Y), 0, st>>>(s->dg, df[0], df[1], df[2], L.dfLB[0],
                                                                           L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
    }
    else if (c6) k_lad_grad<ND, true, true, T><<<gb, 128, 0, st>>>(s->dg, fb, L.fbx, df[0], df[1], df[2], L.dfLB[0], L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
    else k_lad_grad<ND, true, false, T><<<gb, 128, 0, st>>>(s->dg, fb, L.fbx, df[0], df[1], df[2], L.dfLB[0], L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
    k_lad_coef<ND, true, T><<<grid_blocks(s->N, 128), 128, 0, st>>>(s->dg, reinterpret_cast<const T*>(s->W), fb, L.fbx, gr, dv, L.b3, s->p.c_beta,
                                                                    s->p.c_kappa, bt[0], kp[0], guard, want);
  }
  s->launches += 2;
  int cur = 0;
  for (int l = 0; l < ND; ++l) {
    k_gauss<ND, T><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, l, bt[cur], kp[cur], bt[1 - cur], kp[1 - cur],
                                                          guard, want);
    s->launches++;
    cur = 1 - cur;
  }
  if (cur != 0) {
    CG_CUDA(cudaMemcpyAsync(bt[0], bt[1], sizeof(T) * s->N, cudaMemcpyDeviceToDevice, st));
    CG_CUDA(cudaMemcpyAsync(kp[0], kp[1], sizeof(T) * s->N, cudaMemcpyDeviceToDevice, st));
  }
  return CG_OK;
}

template <int ND, int MODE, typename T>
static void lad_nodeflux_m(cg_solver* s, int l, cudaStream_t st, const int* guard, int want, T* out) {
  LadBuffers& L = s->lad;
  int gb = grid_blocks(L.fbox[l].size(), 128);
  const T* bt = reinterpret_cast<const T*>(L.bt[0]);
  const T* kp = reinterpret_cast<const T*>(L.kp[0]);
  const T* gr = reinterpret_cast<const T*>(L.gr);
  const T* dv = reinterpret_cast<const T*>(L.dv);
  T* Fn = out ? out : reinterpret_cast<T*>(L.Fn);
  const T* vco = reinterpret_cast<const T*>(L.vco);
  if (s->dg.curv)
    k_lad_nodeflux<ND, false, MODE, T><<<gb, 128, 0, st>>>(s->dg, l, reinterpret_cast<const T*>(s->W), bt, kp, gr, dv, L.b3, vco, L.vbx, Fn, L.fbox[l], guard, want);
  else
    k_lad_nodeflux<ND, true, MODE, T><<<gb, 128, 0, st>>>(s->dg, l, reinterpret_cast<const T*>(s->W), bt, kp, gr, dv, L.b3, vco, L.vbx, Fn, L.fbox[l], guard, want);
  s->launches++;
}

// mu, lambda, kappa of the physical viscosity at the nodes of every node flux
// (art: with the LAD coefficients beta*, kappa* of bt[0], kp[0])
template <int ND, typename T>
static void lad_viscoef(cg_solver* s, cudaStream_t st, const int* guard, int want, bool art) {
  LadBuffers& L = s->lad;
  const T* W = reinterpret_cast<const T*>(s->W);
  const T* bt = reinterpret_cast<const T*>(L.bt[0]);
  const T* kp = reinterpret_cast<const T*>(L.kp[0]);
  T* vco = reinterpret_cast<T*>(L.vco);
  int gb = grid_blocks(L.vbx.size(), 256);
  if (art) k_lad_viscoef<ND, true, T><<<gb, 256, 0, st>>>(s->dg, W, bt, kp, vco, L.vbx, guard, want);
  else k_lad_viscoef<ND, false, T><<<gb, 256, 0, st>>>(s->dg, W, bt, kp, vco, L.vbx, guard, want);
  s->launches++;
}

// node fluxes along l: mode NF_LAD (artificial terms only), NF_LAD_VISC (plus
// the physical viscosity) or NF_VISC (the physical viscous flux alone)
// (out: where the fluxes go, the shared node-flux buffer when null)
template <int ND, typename T = double>
static void lad_nodeflux(cg_solver* s, int l, cudaStream_t st, const int* guard, int want, int mode = NF_LAD,
                         T* out = nullptr) {
  if (mode == NF_VISC) lad_nodeflux_m<ND, NF_VISC, T>(s, l, st, guard, want, out);
  else if (mode == NF_LAD_VISC) lad_nodeflux_m<ND, NF_LAD_VISC, T>(s, l, st, guard, want, out);
  else lad_nodeflux_m<ND, NF_LAD, T>(s, l, st, guard, want, out);
}

// node fluxes of every direction in one launch (k_lad_nodeflux_all), into out[l]
template <int ND, int MODE, typename T>
static void lad_nodeflux_all_m(cg_solver* s, cudaStream_t st, const int* guard, int want, T* const* out) {
  LadBuffers& L = s->lad;
  const Box& ub = L.ubx;  // [-2, n+1] in every direction
  const int gb = grid_blocks(ub.size(), 128);
  const T* W = reinterpret_cast<const T*>(s->W);
  const T* bt = reinterpret_cast<const T*>(L.bt[0]);
  const T* kp = reinterpret_cast<const T*>(L.kp[0]);
  const T* gr = reinterpret_cast<const T*>(L.gr);
  const T* dv = reinterpret_cast<const T*>(L.dv);
  const T* vco = reinterpret_cast<const T*>(L.vco);
  const Box& f2 = L.fbox[ND == 3 ? 2 : 0];
  if (s->dg.curv)
    k_lad_nodeflux_all<ND, false, MODE, T><<<gb, 128, 0, st>>>(s->dg, W, bt, kp, gr, dv, L.b3, vco, L.vbx, out[0],
                                                               L.fbox[0], out[1], L.fbox[1], out[2], f2, ub, guard, want);
  else
    k_lad_nodeflux_all<ND, true, MODE, T><<<gb, 128, 0, st>>>(s->dg, W, bt, kp, gr, dv, L.b3, vco, L.vbx, out[0],
                                                              L.fbox[0], out[1], L.fbox[1], out[2], f2, ub, guard, want);
  s->launches++;
}

template <int ND, typename T>
static void lad_nodeflux_all(cg_solver* s, cudaStream_t st, const int* guard, int want, int mode, T* const* out) {
  if (mode == NF_LAD_VISC) lad_nodeflux_all_m<ND, NF_LAD_VISC, T>(s, st, guard, want, out);
  else lad_nodeflux_all_m<ND, NF_LAD, T>(s, st, guard, want, out);
}

// E4 gradients of the LAD fields of the primitives in s->W (no coefficients)
template <int ND, typename T>
static void lad_grad_e4(cg_solver* s, cudaStream_t st, const int* guard, int want) {
  LadBuffers& L = s->lad;
  T* fb = reinterpret_cast<T*>(L.fb);
  T* gr = reinterpret_cast<T*>(L.gr);
  T* dv = reinterpret_cast<T*>(L.dv);
  k_lad_fieldbuf<ND, T><<<grid_blocks(L.fbx.size(), 256), 256, 0, st>>>(s->dg, reinterpret_cast<const T*>(s->W), fb, L.fbx);
  int gb = grid_blocks(L.b3.size(), 128);
  if (s->dg.curv)
    k_lad_grad<ND, false, false, T><<<gb, 128, 0, st>>>(s->dg, fb, L.fbx, nullptr, nullptr, nullptr, L.dfLB[0], L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
  else
    k_lad_grad<ND, true, false, T><<<gb, 128, 0, st>>>(s->dg, fb, L.fbx, nullptr, nullptr, nullptr, L.dfLB[0], L.dfLB[1], L.dfLB[2], gr, dv, L.b3, guard, want);
  s->launches += 2;
}

// Physical viscous terms of the C-GBR and per-interface hybrid stages (the
// central viscous routines shared with the LAD framework, no interface
// damping scheme): node fluxes -F^v from E4 gradients of the primitives in
// s->W and their E4 derivative along each direction, accumulated into acc;
// the first direction initialises acc, none runs the epilogue.  have_grad:
// the gradients of this stage's primitives are already in the LAD buffers.
template <int ND, typename T>
static void visc_pass(cg_solver* s, StageArgs A, cudaStream_t st, bool have_grad, const int* guard, int want) {
  LadBuffers& L = s->lad;
  if (!have_grad) lad_grad_e4<ND, T>(s, st, guard, want);
  lad_viscoef<ND, T>(s, st, guard, want, false);
  for (int l = 0; l < ND; ++l) {
    lad_nodeflux<ND, T>(s, l, st, guard, want, NF_VISC);
    A.first = l == 0;
    A.last = false;
    k_lad_div<ND, T><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, l, reinterpret_cast<const T*>(L.Fn), L.fbox[l],
                                                            nullptr, L.DLB[l], A, guard, want);
    s->launches++;
  }
}

template <int ND>
static void visc_pass_any(cg_solver* s, StageArgs A, cudaStream_t st, bool have_grad, const int* guard, int want) {
  if (s->p.precision == CG_MIXED) visc_pass<ND, float>(s, A, st, have_grad, guard, want);
  else visc_pass<ND, double>(s, A, st, have_grad, guard, want);
}

// LAD residual (E4 or C6) of the primitives in s->W with the epilogue of A.
template <int ND, typename T = double>
static int lad_pass(cg_solver* s, int dkind, StageArgs A, cudaStream_t st, const int* guard, int want) {
  int rc = lad_coeffs_run<ND, T>(s, dkind, st, guard, want);
  if (rc) return rc;
  LadBuffers& L = s->lad;
  if (s->p.viscous) lad_viscoef<ND, T>(s, st, guard, want, true);
  const int nfm = s->p.viscous ? NF_LAD_VISC : NF_LAD;
  // C6: every direction's node fluxes and flux lines first (each in its own
  // slice), solved in one launch when all are partitioned; then the divergences
  const T* Dl[3] = {nullptr, nullptr, nullptr};
  if (dkind == 3) {
    LineJob<T> jobs[3];
    const T* Fl[3];
    T* Fw[3] = {nullptr, nullptr, nullptr};
    for (int l = 0; l < ND; ++l) Fw[l] = reinterpret_cast<T*>(L.Fn) + (size_t)l * L.fstride;
    lad_nodeflux_all<ND, T>(s, st, guard, want, nfm, Fw);
    for (int l = 0; l < ND; ++l) {
      Fl[l] = Fw[l];
      T* Dw = reinterpret_cast<T*>(L.D) + (size_t)l * L.dstride;
      jobs[l] = LineJob<T>{&s->c6flux[l], Dw, L.DLB[l].nl, ND + 2};
      Dl[l] = Dw;
    }
    if (rhs_in_solver(jobs, ND)) {  // the solver forms the right-hand sides
      for (int l = 0; l < ND; ++l) jobs[l].src = C6Src<T>{Fl[l], L.fbox[l], L.fbox[l].size(), L.DLB[l]};
      launch_lines(jobs, ND, st);
      s->launches++;
    } else {
      for (int l = 0; l < ND; ++l) {
        launch_rhs_c6<ND, T>(Fl[l], L.fbox[l], ND + 2, L.DLB[l], const_cast<T*>(Dl[l]), st);
        launch_lines(&jobs[l], 1, st);
        s->launches += 2;
      }
    }
  }
  if (ND >= 2 && dkind == 3) {  // all directions' divergences in one tiled pass
    const LineBuf& DL = L.DLB[0];
    const long long ty = (DL.nl + LGT_Y - 1) / LGT_Y;
    const unsigned gy = (unsigned)std::min<long long>(ty, 65535), gz = (unsigned)((ty + gy - 1) / gy);
    if constexpr (ND >= 2)
      k_lad_div_all_xt<ND, T><<<dim3((unsigned)((s->dg.n[0] + LGT_X - 1) / LGT_X), gy, gz), dim3(LGT_X, LGT_Y), 0,
                                st>>>(s->dg, Dl[0], L.DLB[0], Dl[1], L.DLB[1], Dl[2], L.DLB[ND == 3 ? 2 : 1], A, guard,
                                      want);
    s->launches++;
    return CG_OK;
  }
  // E4: every direction's node fluxes in one pass too (slices of Fn)
  T* Fe[3] = {nullptr, nullptr, nullptr};
  if (dkind != 3) {
    for (int l = 0; l < ND; ++l) Fe[l] = reinterpret_cast<T*>(L.Fn) + (size_t)l * L.fstride;
    lad_nodeflux_all<ND, T>(s, st, guard, want, nfm, Fe);
  }
  for (int l = 0; l < ND; ++l) {
    A.first = l == 0;
    A.last = l == ND - 1;
    const T* D = Dl[l];
    LineBuf DL = L.DLB[l];
    if (ND >= 2 && l == 0 && D) {  // x lines: the tiled read of the line buffer
      const long long ty = (DL.nl + LGT_Y - 1) / LGT_Y;
      const unsigned gy = (unsigned)std::min<long long>(ty, 65535), gz = (unsigned)((ty + gy - 1) / gy);
      if constexpr (ND >= 2)
        k_lad_div_xt<ND, T><<<dim3((unsigned)((s->dg.n[0] + LGT_X - 1) / LGT_X), gy, gz), dim3(LGT_X, LGT_Y), 0, st>>>(
            s->dg, D, DL, A, guard, want);
    } else {
      k_lad_div<ND, T><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, l, Fe[l] ? Fe[l] : reinterpret_cast<const T*>(L.Fn),
                                                              L.fbox[l], D, DL, A, guard, want);
    }
    s->launches++;
  }
  return CG_OK;
}

template <int ND, typename T>
static int lad_stage_t(cg_solver* s, const double* Uc, StageArgs A, cudaStream_t st);

template <int ND>
static int lad_stage(cg_solver* s, const double* Uc, StageArgs A, cudaStream_t st) {
  if (s->p.precision == CG_MIXED) return lad_stage_t<ND, float>(s, Uc, A, st);
  return lad_stage_t<ND, double>(s, Uc, A, st);
}

template <int ND, typename T>
static int lad_stage_t(cg_solver* s, const double* Uc, StageArgs A, cudaStream_t st) {
  int sch = s->p.scheme;
  launch_prim<ND>(s, Uc, st);  // T is the precision's type
  if (sch == CG_LAD_E4 || sch == CG_LAD_C6) return lad_pass<ND, T>(s, sch == CG_LAD_E4 ? 2 : 3, A, st, nullptr, 0);
  LadBuffers& L = s->lad;
  CG_CUDA(cudaMemsetAsync(s->hyb_flag, 0, sizeof(int), st));
  CG_CUDA(cudaMemsetAsync(s->hyb_count, 0, sizeof(unsigned long long), st));
  if (s->p.hybrid_mode == CG_HYBRID_GLOBAL) {
    // Algorithm 3: GBR-MEG6 for the whole stage if any node is troubled, else LAD-E4
    k_troubled<ND, T><<<grid_blocks(L.tbox.size(), 256), 256, 0, st>>>(s->dg, reinterpret_cast<const T*>(s->W), s->p.hyb_rho, s->p.hyb_p, nullptr,
                                                                   s->omBox, 0.0, nullptr, L.tbox, s->hyb_flag,
                                                                   s->hyb_count, 0);
    s->launches++;
    stage_prep_gbr<ND>(s, Uc, false, st, false, s->hyb_flag, 1);
    StageArgs G = A;
    G.guard = s->hyb_flag;
    G.guard_want = 1;
    if (s->p.viscous) visc_pass<ND, T>(s, G, st, false, s->hyb_flag, 1);
    int rc = gbr_sweeps<ND>(s, false, G, st, !s->p.viscous);
    if (rc) return rc;
    return lad_pass<ND, T>(s, 2, A, st, s->hyb_flag, 0);
  }
  // per interface: GBR-MEG6 where a neighbour node is troubled, LAD-E4 (flux form) elsewhere
  stage_prep_gbr<ND>(s, Uc, false, st, false);
  k_troubled<ND, T><<<grid_blocks(L.tbox.size(), 256), 256, 0, st>>>(
      s->dg, reinterpret_cast<const T*>(s->W), s->p.hyb_rho, s->p.hyb_p, s->p.hybrid_sensor ? reinterpret_cast<const T*>(s->om) : nullptr, s->omBox, s->p.sensor_thresh, L.tr,
      L.tbox, s->hyb_flag, s->hyb_count, s->p.hybrid_buffer);
  s->launches++;
  int rc = lad_coeffs_run<ND, T>(s, 2, st, nullptr, 0);
  if (rc) return rc;
  if (s->p.viscous) visc_pass<ND, T>(s, A, st, true, nullptr, 0);
  for (int l = 0; l < ND; ++l) {
    lad_nodeflux<ND, T>(s, l, st, nullptr, 0);
    k_lad_hflux<ND, T><<<grid_blocks(L.hbox[l].size(), 256), 256, 0, st>>>(s->dg, l, reinterpret_cast<const T*>(L.Fn),
                                                                          L.fbox[l], reinterpret_cast<T*>(s->hflux[l]), L.hbox[l]);
    s->launches++;
  }
  StageArgs H = A;
  H.mask = L.tr;
  H.tBox = L.tbox;
  for (int d = 0; d < ND; ++d) {
    H.first = d == 0 && !s->p.viscous;
    H.last = d == ND - 1;
    H.hflux = s->hflux[d];
    H.hBox = L.hbox[d];
    H.Gd = nullptr;
    H.gdLB = s->gdLB[d];
    H.iface_out = (s->iface_out && s->iface_dir == d) ? s->iface_out : nullptr;
    if (s->dg.curv) rc = sweep_dir<ND, false, false>(s, d, H, st);
    else rc = sweep_dir<ND, true, false>(s, d, H, st);
    if (rc) return rc;
  }
  return CG_OK;
}

static void filter_coeffs(double af, double b[5]) {
  b[0] = (93.0 + 70.0 * af) / 128.0;
  b[1] = 0.5 * ((7.0 + 18.0 * af) / 16.0);
  b[2] = 0.5 * ((-7.0 + 14.0 * af) / 32.0);
  b[3] = 0.5 * ((1.0 - 2.0 * af) / 16.0);
  b[4] = 0.5 * ((-1.0 + 2.0 * af) / 128.0);
}

template <int ND>
static int lad_filter(cg_solver* s, double* U, cudaStream_t st) {
  if (!s->lad.lines) return fail(CG_ERR_UNSUPPORTED, "the implicit filter belongs to LAD-C6");
  double b[5];
  filter_coeffs(s->p.alpha_f, b);
  if (s->p.precision == CG_MIXED) {  // increment form, FP32 line solves (FilterInc)
    const FilterInc fc{(float)(b[1] - s->p.alpha_f), (float)b[2], (float)b[3], (float)b[4]};
    float* x = reinterpret_cast<float*>(s->lad.lines);
    for (int l = 0; l < ND; ++l) {
      const LineBuf& lb = s->lad.filtLB[l];
      if (use_tile(lb)) {
        using Tl = XTileFilterInc<ND>;
        k_rhs_tile<float, ND + 2, 4, Tl, float2><<<tile_grid(lb), XT_THREADS, 0, st>>>(lb, Tl{s->dg, U, fc, ND + 2}, x);
      } else {
        k_rhs_filter_inc<ND><<<grid_blocks((long long)lb.m * lb.nl, 256), 256, 0, st>>>(s->dg, U, lb, fc, x);
      }
      LineJob<float> job{&s->filt[l], x, lb.nl, ND + 2};
      launch_lines(&job, 1, st);
      if (ND >= 2 && l == 0) {  // x lines: the tiled read of the line buffer
        const long long ty = (lb.nl + FST_Y - 1) / FST_Y;
        const unsigned gy = (unsigned)std::min<long long>(ty, 65535), gz = (unsigned)((ty + gy - 1) / gy);
        k_filter_store_inc_xt<ND><<<dim3((unsigned)((s->dg.n[0] + FST_X - 1) / FST_X), gy, gz), dim3(FST_X, FST_Y), 0,
                                    st>>>(s->dg, x, lb, U);
      } else {
        k_filter_store_inc<ND><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, x, lb, U);
      }
      s->launches += 3;
    }
    return CG_OK;
  }
  for (int l = 0; l < ND; ++l) {
    const LineBuf& lb = s->lad.filtLB[l];
    launch_rhs_filter<ND>(s->dg, U, lb, b, s->lad.lines, st);
    LineJob<double> job{&s->filt[l], s->lad.lines, lb.nl, ND + 2};
    launch_lines(&job, 1, st);
    k_filter_store<ND><<<grid_blocks(s->N, 256), 256, 0, st>>>(s->dg, s->lad.lines, lb, U);
    s->launches += 3;
  }
  return CG_OK;
}

extern "C" {

CG_API int cg_lad_coeffs(cg_solver* s, const double* U, double* beta, double* kappa, void* stream) {
  if (!s || !U || !beta || !kappa) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (!s->lad.gr) return fail(CG_ERR_UNSUPPORTED, "LAD coefficients exist for the LAD and hybrid schemes");
  if (s->p.precision != CG_FP64) return fail(CG_ERR_UNSUPPORTED, "coefficient diagnostics are FP64 only");
  cudaStream_t st = (cudaStream_t)stream;
  DISPATCH_ND(s, stage_prep_prim, s, U, st);
  int rc = DISPATCH_ND(s, lad_coeffs_run, s, s->p.scheme == CG_LAD_C6 ? 3 : 2, st, nullptr, 0);
  if (rc) return rc;
  CG_CUDA(cudaMemcpyAsync(beta, s->lad.bt[0], sizeof(double) * s->N, cudaMemcpyDeviceToDevice, st));
  CG_CUDA(cudaMemcpyAsync(kappa, s->lad.kp[0], sizeof(double) * s->N, cudaMemcpyDeviceToDevice, st));
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_filter(cg_solver* s, double* U, void* stream) {
  if (!s || !U) return fail(CG_ERR_INVALID_ARG, "null argument");
  int rc = DISPATCH_ND(s, lad_filter, s, U, (cudaStream_t)stream);
  if (rc) return rc;
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

CG_API int cg_hybrid_state(cg_solver* s, int* last_flag, int64_t* n_troubled, void* stream) {
  if (!s) return fail(CG_ERR_INVALID_ARG, "null argument");
  if (s->p.scheme != CG_HYBRID) return fail(CG_ERR_UNSUPPORTED, "not a hybrid solver");
  cudaStream_t st = (cudaStream_t)stream;
  int f = 0;
  unsigned long long c = 0;
  CG_CUDA(cudaMemcpyAsync(&f, s->hyb_flag, sizeof f, cudaMemcpyDeviceToHost, st));
  CG_CUDA(cudaMemcpyAsync(&c, s->hyb_count, sizeof c, cudaMemcpyDeviceToHost, st));
  CG_CUDA(cudaStreamSynchronize(st));
  if (last_flag) *last_flag = f;
  if (n_troubled) *n_troubled = (int64_t)c;
  return CG_OK;
}

}  // extern "C"
