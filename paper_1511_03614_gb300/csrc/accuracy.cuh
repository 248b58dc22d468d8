// accuracy.cuh -- the flow proposal inside fiesta_integrate, and the accuracy loops of
// fiesta_integrate_to_accuracy (included at the end of fiesta.cu; host code).
//
// The paper's pool integrates, checks the error against the requested accuracy and
// continues (Sec. 4.5-4.6); here that loop runs inside the library on top of the
// integration entry points: per-result inverse-variance combination of iterations
// across calls, the per-order sums with mean-square errors (Sec. 4.3), the eps-series
// prefactor, the per-order target check, Neyman allocation of points across units,
// the replicate statistics of randomised quasi-Monte Carlo, the flow's training
// rounds and the cubature's tolerance schedule.

namespace {

struct RecInfo {
    int64_t unit;
    int out;      // result index within the unit
    int order;    // eps order
    int part;     // 0 real, 1 imaginary part of a complex unit
};

std::vector<RecInfo> all_records(const fiesta_ctx *c) {
    std::vector<RecInfo> r;
    for (int64_t k = 0; k < (int64_t)c->units.size(); ++k) {
        const DevUnit &u = c->units[k];
        for (int o = 0; o < u.n_out; ++o) r.push_back({k, o, u.order + (u.cplx ? o / 2 : o), u.cplx ? (o & 1) : 0});
    }
    return r;
}

// The assembled series R_n = sum_i c_i I_(n - (i - q)) of per-order sums I_K over
// records, for n = out_lo .. out_lo + n_out - 1; real and imaginary parts separately.
// Per-order errors: sqrt(sum sigma^2) (independent results) or sum sigma (bounds,
// `linear`); through the prefactor: sum |c_i| E (correlated orders) or
// sqrt(sum c_i^2 E^2).
struct Series {
    std::vector<double> re, im, ere, eim;
};

Series assemble_arrays(int64_t n_rec, const int32_t *order, const int32_t *part, const double *val,
                       const double *sig, const fiesta_accuracy_options *o, int n_out, bool linear) {
    int kmin = 1 << 30, kmax = -(1 << 30);
    for (int64_t k = 0; k < n_rec; ++k) {
        kmin = std::min(kmin, order[k]);
        kmax = std::max(kmax, order[k]);
    }
    const int nk = std::max(kmax - kmin + 1, 0);
    std::vector<double> I[2] = {std::vector<double>(nk, 0.0), std::vector<double>(nk, 0.0)};
    std::vector<double> E[2] = {std::vector<double>(nk, 0.0), std::vector<double>(nk, 0.0)};
    for (int64_t k = 0; k < n_rec; ++k) {
        const int K = order[k] - kmin, p = part[k] ? 1 : 0;
        I[p][K] += val[k];
        E[p][K] += linear ? sig[k] : sig[k] * sig[k];
    }
    if (!linear)
        for (int p = 0; p < 2; ++p)
            for (double &e : E[p]) e = std::sqrt(e);
    Series S;
    S.re.assign(n_out, 0.0);
    S.im.assign(n_out, 0.0);
    S.ere.assign(n_out, 0.0);
    S.eim.assign(n_out, 0.0);
    const bool lin = linear || o->correlated;
    for (int n = 0; n < n_out; ++n) {
        const int ord = o->out_lo + n;
        double v[2] = {0.0, 0.0}, e1[2] = {0.0, 0.0}, e2[2] = {0.0, 0.0};
        for (int i = 0; i < o->n_pre; ++i) {
            const int K = ord - (i - o->pre_q) - kmin;
            if (K < 0 || K >= nk) continue;
            const double ci = o->pre[i];
            for (int p = 0; p < 2; ++p) {
                v[p] += ci * I[p][K];
                e1[p] += std::fabs(ci) * E[p][K];
                e2[p] += ci * ci * E[p][K] * E[p][K];
            }
        }
        S.re[n] = v[0];
        S.im[n] = v[1];
        S.ere[n] = lin ? e1[0] : std::sqrt(e2[0]);
        S.eim[n] = lin ? e1[1] : std::sqrt(e2[1]);
    }
    return S;
}

Series assemble_series(const std::vector<RecInfo> &recs, const double *val, const double *sig,
                       const fiesta_accuracy_options *o, int n_out, bool linear) {
    std::vector<int32_t> order(recs.size()), part(recs.size());
    for (size_t k = 0; k < recs.size(); ++k) {
        order[k] = recs[k].order;
        part[k] = recs[k].part;
    }
    return assemble_arrays((int64_t)recs.size(), order.data(), part.data(), val, sig, o, n_out, linear);
}

// max over orders of |E_n| / (target * max(|R_n|, floor * max_k |R_k|)) (moduli of
// (re, im) pairs).
double worst_ratio(const Series &S, double target, double floor_) {
    double big = 0.0;
    for (size_t n = 0; n < S.re.size(); ++n) big = std::max(big, std::hypot(S.re[n], S.im[n]));
    double worst = 0.0;
    for (size_t n = 0; n < S.re.size(); ++n) {
        const double tau = target * std::max(std::hypot(S.re[n], S.im[n]), floor_ * big);
        const double e = std::hypot(S.ere[n], S.eim[n]);
        worst = std::max(worst, tau > 0.0 ? e / tau : (e > 0.0 ? HUGE_VAL : 0.0));
    }
    return worst;
}

// Neyman allocation for the assembled series: unit u's per-point spread of its order-K
// integral is s_uK = sigma_uK sqrt(points used); its share of the error of order n is
// sum_K |c_(n-K)| s_uK / sqrt(N_u); with B_u = max_n (sum_K |c_(n-K)| s_uK / tau_n)^2
// and the cost per point w_u, N_u proportional to sqrt(B_u / w_u) minimises the cost
// at a given error.  The total cost equals that of `points` per unit; each N_u lies
// in [max(2, 0.01 points), 64 points].
void neyman_arrays(const fiesta_accuracy_options *o, int64_t nu, const double *cost, int64_t n_rec,
                   const int64_t *rec_unit, const int32_t *rec_order, const double *sig, const double *n_used,
                   int n_out, const double *re, const double *im, int64_t *N) {
    const double points = (double)o->points;
    double big = 0.0;
    for (int n = 0; n < n_out; ++n) big = std::max(big, std::hypot(re[n], im ? im[n] : 0.0));
    std::vector<double> tau(n_out);
    for (int n = 0; n < n_out; ++n) tau[n] = o->target * std::max(std::hypot(re[n], im ? im[n] : 0.0), o->floor * big);
    int kmin = 1 << 30, kmax = -(1 << 30);
    for (int64_t k = 0; k < n_rec; ++k) {
        kmin = std::min(kmin, rec_order[k]);
        kmax = std::max(kmax, rec_order[k]);
    }
    const int nk = std::max(kmax - kmin + 1, 1);
    std::vector<double> s2((size_t)nu * nk, 0.0);
    for (int64_t k = 0; k < n_rec; ++k)
        s2[rec_unit[k] * nk + rec_order[k] - kmin] += sig[k] * sig[k] * n_used[rec_unit[k]];
    std::vector<double> wgt(nu);
    double csum = 0.0, wc = 0.0;
    bool any = false;
    for (int64_t u = 0; u < nu; ++u) {
        double B = 0.0;
        for (int n = 0; n < n_out; ++n) {
            double acc = 0.0;
            for (int K = 0; K < nk; ++K) {
                const int i = (o->out_lo + n) - (K + kmin) + o->pre_q;
                if (i >= 0 && i < o->n_pre) acc += std::fabs(o->pre[i]) * std::sqrt(s2[u * nk + K]);
            }
            if (tau[n] > 0.0) B = std::max(B, (acc / tau[n]) * (acc / tau[n]));
        }
        wgt[u] = std::sqrt(std::max(B, 0.0) / cost[u]);
        any = any || wgt[u] > 0.0;
        csum += cost[u];
        wc += wgt[u] * cost[u];
    }
    for (int64_t u = 0; u < nu; ++u) {
        if (!any) {
            N[u] = o->points;
            continue;
        }
        double x = wgt[u] * points * csum / wc;
        x = std::min(std::max(x, std::max(2.0, 0.01 * points)), 64.0 * points);
        N[u] = std::max<int64_t>((int64_t)x, 2);
    }
}

std::vector<int64_t> neyman(const fiesta_ctx *c, const std::vector<RecInfo> &recs, const double *sig,
                            const double *n_used, const Series &S, const fiesta_accuracy_options *o) {
    const int64_t nu = (int64_t)c->units.size();
    std::vector<double> cost(nu);
    for (int64_t u = 0; u < nu; ++u) cost[u] = c->units[u].n_instr + 4.0 * c->units[u].dim + 8.0;
    std::vector<int64_t> ru(recs.size()), N(nu);
    std::vector<int32_t> ro(recs.size());
    for (size_t k = 0; k < recs.size(); ++k) {
        ru[k] = recs[k].unit;
        ro[k] = recs[k].order;
    }
    neyman_arrays(o, nu, cost.data(), (int64_t)recs.size(), ru.data(), ro.data(), sig, n_used, (int)S.re.size(),
                  S.re.data(), S.im.data(), N.data());
    return N;
}

void write_outputs(const Series &S, const std::vector<RecInfo> &recs, const fiesta_accuracy_state *st, int n_out,
                   double *value, double *error, double *value_im, double *error_im, double *unit_value,
                   double *unit_sigma) {
    for (int n = 0; n < n_out; ++n) {
        value[n] = S.re[n];
        error[n] = S.ere[n];
        if (value_im) value_im[n] = S.im[n];
        if (error_im) error_im[n] = S.eim[n];
    }
    for (size_t k = 0; k < recs.size(); ++k) {
        const double sw = st->sw[k];
        if (unit_value) unit_value[k] = sw > 0.0 ? st->swi[k] / sw : 0.0;
        if (unit_sigma) unit_sigma[k] = sw > 0.0 ? std::sqrt(1.0 / sw) : HUGE_VAL;
    }
}

// Current estimates of every record from the running sums.
void estimates(const fiesta_accuracy_state *st, size_t n, std::vector<double> &val, std::vector<double> &sig) {
    val.resize(n);
    sig.resize(n);
    for (size_t k = 0; k < n; ++k) {
        val[k] = st->sw[k] > 0.0 ? st->swi[k] / st->sw[k] : 0.0;
        sig[k] = st->sw[k] > 0.0 ? std::sqrt(1.0 / st->sw[k]) : HUGE_VAL;
    }
}

// Per-iteration (mean, variance) of record k of the last fiesta_integrate call.
inline void iteration_of(const fiesta_ctx *c, const RecInfo &r, int it, double &m, double &v) {
    const int64_t ko = (r.unit - c->last_begin) * c->last_ostride + r.out;
    m = c->h_iter_mean[ko * c->last_iters + it];
    v = c->h_iter_var[ko * c->last_iters + it];
}

fiesta_options base_options(const fiesta_accuracy_options *o) {
    fiesta_options f;
    std::memset(&f, 0, sizeof(f));
    f.rng = FIESTA_RNG_PHILOX;
    f.precision = o->precision;
    f.n_iter = 1;
    f.adapt = 2;
    f.points_per_iter = o->points;
    f.seed = o->seed;
    f.alpha = 1.5;
    f.small_x = o->small_x;
    f.small_x32 = o->small_x32;
    return f;
}

int64_t unit_evaluations(const fiesta_ctx *c, int64_t points) {
    int64_t n = 0;
    for (const DevUnit &u : c->units) n += points * (u.cplx ? u.n_out / 2 : u.n_out);
    return n;
}

// The flow proposal of fiesta_integrate: each iteration is one pass of the flow
// sampler; between iterations the flows train on points kept from it.
int integrate_flow(fiesta_ctx *c, const fiesta_options *opt, double *value, double *error, int32_t n_orders,
                   fiesta_unit_result *per_unit, fiesta_stats *stats) {
    if (opt->n_iter < 1 || opt->points_per_iter < 2)
        return fail(FIESTA_E_INVALID, "fiesta_integrate: need n_iter >= 1 and points_per_iter >= 2");
    if (opt->precision != FIESTA_FP64 && opt->precision != FIESTA_FP32)
        return fail(FIESTA_E_INVALID, "fiesta_integrate: the flow proposal evaluates in FIESTA_FP64 or FIESTA_FP32");
    if (opt->unit_points) return fail(FIESTA_E_INVALID, "fiesta_integrate: unit_points does not apply to the flow proposal");
    if (opt->flow_train_steps < 0 || opt->flow_keep < 0 || opt->flow_lr < 0.0 || opt->flow_power < 0)
        return fail(FIESTA_E_INVALID, "fiesta_integrate: bad flow training parameters");
    const int64_t total = (int64_t)c->units.size();
    const int64_t b = opt->unit_begin, e = opt->unit_end <= 0 ? total : opt->unit_end;
    if (b < 0 || e > total || b >= e) return fail(FIESTA_E_INVALID, "fiesta_integrate: bad unit slice");
    const int n_iter = opt->n_iter;
    const int64_t N = opt->points_per_iter, nu = e - b;
    const int64_t keep = std::min<int64_t>(opt->flow_keep > 0 ? opt->flow_keep : 4096, N);
    const int steps = opt->flow_train_steps;
    const double lr = opt->flow_lr > 0.0 ? opt->flow_lr : 2e-3;
    const int power = opt->flow_power > 0 ? opt->flow_power : 1;
    if (!c->flow) {
        int r = fiesta_flow_init(c, opt->seed, 0.05);
        if (r) return r;
    }
    const SliceInfo si = slice_info(c, b, e);
    const int ostride = si.max_out;
    int64_t nrec = 0;
    for (int64_t k = b; k < e; ++k) nrec += c->units[k].n_out;
    std::vector<double> mean((size_t)nu * ostride * n_iter, 0.0), var(mean.size(), 0.0);
    std::vector<unsigned long long> ubad(nu, 0), bad_now(nu);
    std::vector<double> m(nrec), v(nrec);
    double total_ms = 0.0, eval_ms = 0.0;
    int launches = 0, eval_launches = 0;
    for (int it = 0; it < n_iter; ++it) {
        fiesta_stats st;
        std::memset(&st, 0, sizeof(st));
        const bool train = steps > 0 && it + 1 < n_iter;
        int r = fiesta_flow_sample(c, b, e, N, opt->seed, opt->iter_offset + it, opt->precision, train ? keep : 0,
                                   m.data(), v.data(), &st);
        if (r && r != FIESTA_E_NONFINITE) return r;
        CUDA_TRY(cudaMemcpy(bad_now.data(), c->d_unit_bad, sizeof(unsigned long long) * nu, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < nu; ++k) ubad[k] += bad_now[k];
        total_ms += st.gpu_ms;
        eval_ms += st.eval_ms;
        launches += st.kernels_launched;
        eval_launches += st.eval_launches;
        int64_t rec = 0;
        for (int64_t k = 0; k < nu; ++k)
            for (int o = 0; o < c->units[b + k].n_out; ++o, ++rec) {
                mean[(k * ostride + o) * n_iter + it] = m[rec];
                var[(k * ostride + o) * n_iter + it] = v[rec];
            }
        if (train) {
            fiesta_stats s2;
            std::memset(&s2, 0, sizeof(s2));
            r = fiesta_flow_train(c, b, e, steps, lr, power, nullptr, &s2);
            if (r) return r;
            total_ms += s2.gpu_ms;
            launches += s2.kernels_launched;
        }
    }
    std::vector<int> fp32(nu, opt->precision == FIESTA_FP32 ? 1 : 0);
    std::vector<double> perr(nu, std::nan(""));
    CallReport R;
    R.b = b;
    R.nu = nu;
    R.ostride = ostride;
    R.n_iter = n_iter;
    R.mean = &mean;
    R.var = &var;
    R.ubad = &ubad;
    R.fp32 = &fp32;
    R.perr = &perr;
    R.N = N;
    R.skip_first = opt->skip_first;
    R.order_lo = opt->order_lo;
    R.total_ms = total_ms;
    R.eval_ms = eval_ms;
    R.launches = launches;
    R.eval_launches = eval_launches;
    R.n32 = opt->precision == FIESTA_FP32 ? nu : 0;
    return report_call(c, R, value, error, n_orders, per_unit, stats);
}

}  // namespace

extern "C" int fiesta_integrate_to_accuracy(fiesta_ctx *c, const fiesta_accuracy_options *o,
                                            fiesta_accuracy_state *st, int32_t n_out, double *value, double *error,
                                            double *value_im, double *error_im, double *unit_value,
                                            double *unit_sigma) {
    if (!c || !o || !st || !st->sw || !st->swi || !st->n_used || n_out < 1 || !value || !error)
        return fail(FIESTA_E_INVALID, "fiesta_integrate_to_accuracy: null argument");
    if (!(o->target > 0.0) || !(o->floor >= 0.0) || o->points < 2 || o->max_iters < 1 || o->skip < 0 ||
        o->n_pre < 1 || !o->pre || o->max_calls < 0 || !(o->max_gpu_s >= 0.0))
        return fail(FIESTA_E_INVALID, "fiesta_integrate_to_accuracy: bad options");
    const std::vector<RecInfo> recs = all_records(c);
    const size_t nrec = recs.size();
    std::vector<double> val, sig;
    const auto capped = [&]() { return o->max_gpu_s > 0.0 && st->gpu_ms * 1e-3 >= o->max_gpu_s; };
    // RQMC with per-order sums: the assembled values and errors come from them
    const bool per_order = o->method == FIESTA_METHOD_RQMC && st->order_sw && st->order_swi;
    const auto check = [&](bool linear) {
        estimates(st, nrec, val, sig);
        Series S = assemble_series(recs, val.data(), sig.data(), o, n_out, linear);
        if (per_order)
            for (int n = 0; n < n_out; ++n) {
                const double w = st->order_sw[n], wi = st->order_sw[n_out + n];
                S.re[n] = w > 0.0 ? st->order_swi[n] / w : 0.0;
                S.ere[n] = w > 0.0 ? std::sqrt(1.0 / w) : HUGE_VAL;
                S.im[n] = wi > 0.0 ? st->order_swi[n_out + n] / wi : 0.0;
                S.eim[n] = wi > 0.0 ? std::sqrt(1.0 / wi) : 0.0;
            }
        st->ratio = worst_ratio(S, o->target, o->floor);
        st->converged = st->ratio <= 1.0 ? 1 : 0;
        write_outputs(S, recs, st, n_out, value, error, value_im, error_im, unit_value, unit_sigma);
        return S;
    };

    if (o->method == FIESTA_METHOD_VEGAS && o->proposal == FIESTA_PROPOSAL_FLOW) {
        if (o->precision != FIESTA_FP64 && o->precision != FIESTA_FP32)
            return fail(FIESTA_E_INVALID, "fiesta_integrate_to_accuracy: the flow proposal needs FP64 or FP32");
        const int train_rounds = o->train_rounds > 0 ? o->train_rounds : 8;
        const int steps = o->steps_per_round > 0 ? o->steps_per_round : 20;
        const double lr = o->lr > 0.0 ? o->lr : 2e-3;
        const int power = o->power > 0 ? o->power : 1;
        const int64_t keep = std::min<int64_t>(o->keep > 0 ? o->keep : 4096, o->points);
        if (st->iterations == 0) {
            int r = fiesta_flow_init(c, o->seed, 0.05);
            if (r) return r;
        }
        std::vector<double> m(nrec), v(nrec);
        int calls = 0;
        for (int rnd = st->iterations; rnd < o->max_iters; ++rnd) {
            fiesta_stats s1;
            std::memset(&s1, 0, sizeof(s1));
            int r = fiesta_flow_sample(c, 0, (int64_t)c->units.size(), o->points, o->seed, rnd, o->precision,
                                       rnd < train_rounds ? keep : 0, m.data(), v.data(), &s1);
            if (r) return r;
            st->gpu_ms += s1.gpu_ms;
            st->points += unit_evaluations(c, o->points);
            if (rnd >= o->skip)
                for (size_t k = 0; k < nrec; ++k) {
                    const double w = v[k] > 0.0 ? 1.0 / v[k] : 1e300;
                    st->sw[k] += w;
                    st->swi[k] += w * m[k];
                }
            if (rnd < train_rounds) {
                fiesta_stats s2;
                std::memset(&s2, 0, sizeof(s2));
                r = fiesta_flow_train(c, 0, (int64_t)c->units.size(), steps, lr, power, nullptr, &s2);
                if (r) return r;
                st->gpu_ms += s2.gpu_ms;
            }
            st->iterations = rnd + 1;
            ++calls;
            if (rnd < o->skip) continue;
            check(false);
            if ((st->converged && rnd >= train_rounds) || capped() || (o->max_calls && calls >= o->max_calls)) break;
        }
        return FIESTA_OK;
    }

    if (o->method == FIESTA_METHOD_VEGAS) {
        if (o->proposal != FIESTA_PROPOSAL_VEGAS) return fail(FIESTA_E_INVALID, "fiesta_integrate_to_accuracy: unknown proposal");
        const int ipc = o->iters_per_call > 0 ? o->iters_per_call : 2;
        std::vector<int64_t> up;          // per-unit points of the next call (empty: o->points each)
        int calls = 0;
        while (st->iterations < o->max_iters) {
            fiesta_options f = base_options(o);
            f.n_iter = ipc;
            f.reset_grid = st->iterations == 0 ? 1 : 0;
            f.iter_offset = st->iterations;
            f.unit_points = up.empty() ? nullptr : up.data();
            fiesta_stats s1;
            std::memset(&s1, 0, sizeof(s1));
            int r = fiesta_integrate(c, &f, nullptr, nullptr, 0, nullptr, &s1);
            if (r) return r;
            st->gpu_ms += s1.gpu_ms;
            st->points += s1.unit_points;
            const int it = st->iterations;
            int counted = 0;
            for (int j = 0; j < ipc; ++j) counted += (it + j >= o->skip) ? 1 : 0;
            for (int64_t u = 0; u < (int64_t)c->units.size(); ++u)
                st->n_used[u] += (double)(up.empty() ? o->points : up[u]) * counted;
            for (size_t k = 0; k < nrec; ++k)
                for (int j = 0; j < ipc; ++j) {
                    if (it + j < o->skip) continue;
                    double m, v;
                    iteration_of(c, recs[k], j, m, v);
                    const double w = v > 0.0 ? 1.0 / v : 1e300;
                    st->sw[k] += w;
                    st->swi[k] += w * m;
                }
            st->iterations += ipc;
            ++calls;
            if (st->iterations <= o->skip) {
                if (o->max_calls && calls >= o->max_calls) break;
                continue;
            }
            const Series S = check(false);
            if (st->converged || capped() || (o->max_calls && calls >= o->max_calls)) break;
            if (o->allocate) {
                bool all_used = true;
                for (int64_t u = 0; u < (int64_t)c->units.size(); ++u) all_used = all_used && st->n_used[u] > 0.0;
                if (all_used) up = neyman(c, recs, sig.data(), st->n_used, S, o);
            }
        }
        return FIESTA_OK;
    }

    if (o->method == FIESTA_METHOD_RQMC) {
        const int R = o->replicates > 0 ? o->replicates : 8;
        if (R < 2) return fail(FIESTA_E_INVALID, "fiesta_integrate_to_accuracy: randomised QMC needs >= 2 replicates");
        const int64_t max_points = o->max_points > 0 ? o->max_points : (int64_t(1) << 22);
        if (st->iterations == 0) {
            fiesta_options f = base_options(o);
            f.n_iter = o->adapt_iters > 0 ? o->adapt_iters : 6;
            f.points_per_iter = o->adapt_points > 0 ? o->adapt_points : o->points;
            f.reset_grid = 1;
            fiesta_stats s1;
            std::memset(&s1, 0, sizeof(s1));
            int r = fiesta_integrate(c, &f, nullptr, nullptr, 0, nullptr, &s1);
            if (r) return r;
            st->gpu_ms += s1.gpu_ms;
            st->points += s1.unit_points;
        }
        int64_t n = st->points_per_replicate > 0 ? 2 * st->points_per_replicate : o->points;
        for (int rnd = st->iterations; rnd < o->max_iters; ++rnd) {
            fiesta_options f = base_options(o);
            f.rng = FIESTA_RNG_SOBOL;
            f.n_iter = R;
            f.points_per_iter = n;
            f.seed = o->seed + 1 + rnd;
            f.adapt = 0;
            f.iter_offset = 1000 + rnd * R;
            fiesta_stats s1;
            std::memset(&s1, 0, sizeof(s1));
            int r = fiesta_integrate(c, &f, nullptr, nullptr, 0, nullptr, &s1);
            if (r) return r;
            st->gpu_ms += s1.gpu_ms;
            st->points += s1.unit_points;
            for (size_t k = 0; k < nrec; ++k) {
                double mu = 0.0, m, v;
                for (int j = 0; j < R; ++j) {
                    iteration_of(c, recs[k], j, m, v);
                    mu += m;
                }
                mu /= R;
                double ss = 0.0;
                for (int j = 0; j < R; ++j) {
                    iteration_of(c, recs[k], j, m, v);
                    ss += (m - mu) * (m - mu);
                }
                const double var = ss / (R - 1) / R;
                const double w = var > 0.0 ? 1.0 / var : 1e300;
                st->sw[k] += w;
                st->swi[k] += w * mu;
            }
            if (per_order) {
                // the assembled series of every replicate (its records' replicate means
                // through the prefactor), then per order the replicate mean and spread
                std::vector<double> mj(nrec), zero(nrec, 0.0);
                std::vector<double> a_re((size_t)R * n_out), a_im((size_t)R * n_out);
                for (int j = 0; j < R; ++j) {
                    for (size_t k = 0; k < nrec; ++k) {
                        double m, v;
                        iteration_of(c, recs[k], j, m, v);
                        mj[k] = m;
                    }
                    const Series A = assemble_series(recs, mj.data(), zero.data(), o, n_out, false);
                    for (int n = 0; n < n_out; ++n) {
                        a_re[(size_t)j * n_out + n] = A.re[n];
                        a_im[(size_t)j * n_out + n] = A.im[n];
                    }
                }
                for (int p = 0; p < 2; ++p) {
                    const std::vector<double> &a = p ? a_im : a_re;
                    for (int n = 0; n < n_out; ++n) {
                        double mu = 0.0, ss = 0.0;
                        for (int j = 0; j < R; ++j) mu += a[(size_t)j * n_out + n];
                        mu /= R;
                        for (int j = 0; j < R; ++j) {
                            const double d = a[(size_t)j * n_out + n] - mu;
                            ss += d * d;
                        }
                        const double var = ss / (R - 1) / R;
                        if (p && var == 0.0 && mu == 0.0) continue;       // no imaginary part
                        const double w = var > 0.0 ? 1.0 / var : 1e300;
                        st->order_sw[p * n_out + n] += w;
                        st->order_swi[p * n_out + n] += w * mu;
                    }
                }
            }
            st->points_per_replicate = n;
            st->iterations = rnd + 1;
            check(false);
            if (st->converged || 2 * n > max_points || capped()) break;
            n *= 2;
        }
        return FIESTA_OK;
    }

    if (o->method == FIESTA_METHOD_CUHRE) {
        double tol = st->rel_tol > 0.0 ? st->rel_tol * (o->shrink > 0.0 ? o->shrink : 0.1)
                                       : (o->rel_tol > 0.0 ? o->rel_tol : o->target);
        std::vector<fiesta_cuhre_result> res(nrec);
        for (int attempt = st->iterations; attempt < o->max_iters; ++attempt) {
            fiesta_cuhre_options co;
            std::memset(&co, 0, sizeof(co));
            co.rel_tol = tol;
            co.abs_tol = 1e-12;
            co.max_passes = o->max_passes > 0 ? o->max_passes : 60;
            co.max_regions = o->max_regions > 0 ? o->max_regions : (int64_t(1) << 22);
            fiesta_stats s1;
            std::memset(&s1, 0, sizeof(s1));
            int r = fiesta_cuhre(c, &co, nullptr, nullptr, 0, res.data(), &s1);
            if (r) return r;
            st->gpu_ms += s1.gpu_ms;
            st->points += s1.points;
            // the latest attempt replaces the estimates: bounds, not samples to average
            for (size_t k = 0; k < nrec; ++k) {
                st->sw[k] = res[k].error > 0.0 ? 1.0 / (res[k].error * res[k].error) : 1e300;
                st->swi[k] = st->sw[k] * res[k].value;
            }
            st->rel_tol = tol;
            st->iterations = attempt + 1;
            std::vector<double> v(nrec), e(nrec);
            for (size_t k = 0; k < nrec; ++k) {
                v[k] = res[k].value;
                e[k] = res[k].error;
            }
            const Series S = assemble_series(recs, v.data(), e.data(), o, n_out, true);
            st->ratio = worst_ratio(S, o->target, o->floor);
            st->converged = st->ratio <= 1.0 ? 1 : 0;
            write_outputs(S, recs, st, n_out, value, error, value_im, error_im, nullptr, nullptr);
            if (unit_value)
                for (size_t k = 0; k < nrec; ++k) unit_value[k] = v[k];
            if (unit_sigma)
                for (size_t k = 0; k < nrec; ++k) unit_sigma[k] = e[k];
            if (st->converged || capped()) break;
            tol *= o->shrink > 0.0 ? o->shrink : 0.1;
        }
        return FIESTA_OK;
    }
    return fail(FIESTA_E_INVALID, "fiesta_integrate_to_accuracy: unknown method");
}

extern "C" int fiesta_assemble(const fiesta_accuracy_options *o, int64_t n_rec, const int32_t *order,
                               const int32_t *part, const double *val, const double *sig, int32_t linear,
                               int32_t n_out, double *value, double *error, double *value_im, double *error_im,
                               double *ratio) {
    if (!o || n_rec < 1 || !order || !part || !val || !sig || n_out < 1 || !value || !error || !o->pre ||
        o->n_pre < 1)
        return fail(FIESTA_E_INVALID, "fiesta_assemble: bad arguments");
    const Series S = assemble_arrays(n_rec, order, part, val, sig, o, n_out, linear != 0);
    for (int n = 0; n < n_out; ++n) {
        value[n] = S.re[n];
        error[n] = S.ere[n];
        if (value_im) value_im[n] = S.im[n];
        if (error_im) error_im[n] = S.eim[n];
    }
    if (ratio) *ratio = worst_ratio(S, o->target, o->floor);
    return FIESTA_OK;
}

extern "C" int fiesta_allocate_points(const fiesta_accuracy_options *o, int64_t n_units, const double *cost,
                                      int64_t n_rec, const int64_t *rec_unit, const int32_t *rec_order,
                                      const double *sig, const double *n_used, int32_t n_out, const double *value,
                                      const double *value_im, int64_t *points) {
    if (!o || n_units < 1 || !cost || n_rec < 1 || !rec_unit || !rec_order || !sig || !n_used || n_out < 1 ||
        !value || !points || !o->pre || o->n_pre < 1 || o->points < 2)
        return fail(FIESTA_E_INVALID, "fiesta_allocate_points: bad arguments");
    for (int64_t k = 0; k < n_rec; ++k)
        if (rec_unit[k] < 0 || rec_unit[k] >= n_units) return fail(FIESTA_E_INVALID, "fiesta_allocate_points: bad record unit");
    for (int64_t u = 0; u < n_units; ++u)
        if (!(cost[u] > 0.0)) return fail(FIESTA_E_INVALID, "fiesta_allocate_points: costs must be > 0");
    neyman_arrays(o, n_units, cost, n_rec, rec_unit, rec_order, sig, n_used, n_out, value, value_im, points);
    return FIESTA_OK;
}
