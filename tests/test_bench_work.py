"""bench.py's algorithmic-work model: every modelled kernel has positive work
on the benchmark workload, the fused layout moves the prediction sweep's rows
into the fit's sweep, and the sweep's update is split between the
super-panel kernel and the panel steps without double counting."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_work_model_c2():
    import bench
    from workloads import make_problem
    p = make_problem("C2", B=1)
    fused = bench.kernel_work(p, 1, fused=True)
    plain = bench.kernel_work(p, 1, fused=False)
    assert all(v > 0 for v in fused.values())
    assert "k_pred_sweep_tc" not in fused and plain["k_pred_sweep_tc"] > 0
    # the test rows add work to the fit's sweep only
    for k in ("k_chol_panel_pt", "k_chol_wide", "k_chol_mid"):
        assert fused[k] > plain[k]
    for k in ("k_resid_bf6", "k_gram_bf6", "k_pred_rhs_bf6", "k_proj", "k_f64_chain"):
        assert fused[k] == plain[k]
    # left-looking update of the windows, counted once: wide + mid + step = the full left-looking sum
    s = p.s
    full = 0.0
    for n, b, nb in bench.window_sizes(p.block_ptr, 1):
        rows = n + s + 1
        for k0 in range(0, n, 64):
            w = min(64, n - k0)
            full += 2.0 * ((rows - k0) * w - w * (w - 1) / 2.0) * k0
    tri = 0.0
    for n, b, nb in bench.window_sizes(p.block_ptr, 1):
        rows = n + s + 1
        for k0 in range(0, n, 64):
            w = min(64, n - k0)
            tri += max(0, rows - k0 - w) * w * w
    # the persistent panel kernel's update of the rows below each diagonal
    # block plus the diagonal blocks' own update (64 x 64 lower triangles,
    # K = k0 - kh, left to k_chol_step_tc) complete the sum
    diag = 0.0
    for n, b, nb in bench.window_sizes(p.block_ptr, 1):
        for k0 in range(0, n, 64):
            w = min(64, n - k0)
            diag += 2.0 * (w * w - w * (w - 1) / 2.0) * (k0 - (k0 // 128) * 128)
    panel_update = plain["k_chol_panel_pt"] - tri
    assert abs(plain["k_chol_wide"] + plain["k_chol_mid"] + panel_update + diag - full) <= 1e-9 * full
