"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/paradiag.h declares (CPU only, no compute calls)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "paradiag.h")).read()
    return re.findall(r"PD_API\s+[\w\s\*]+?\b(pd[1hc]?_\w+)\s*\(", txt)


def test_header_declares_the_boundary():
    names = set(header_symbols())
    for n in ("pd_plan_create", "pd_plan_destroy", "pd_apply_precond", "pd_residual",
              "pd_apply_A", "pd_build_rhs", "pd_solve", "pd_adjoint_solve"):
        assert n in names


def test_library_exports_every_header_symbol():
    import paradiag_gb300 as pd
    pd.build()
    lib = pd.load()
    names = header_symbols()
    assert names
    for n in names:
        assert hasattr(lib, n), n
    # the Python binding exposes the same names
    for n in names:
        assert hasattr(pd, n), n


def test_status_strings_without_gpu():
    import paradiag_gb300 as pd
    pd.build()
    assert pd.pd_status_string(0) == "ok"
    assert pd.pd_status_string(-5) == "unsupported problem"


def test_plan_create_rejects_bad_arguments_without_gpu():
    # argument validation happens before any CUDA call
    import paradiag_gb300 as pd
    pd.build()
    sp = pd.pd_space(1, 15, 1, 0.1, 0.0, 0.0, 0, 0, 1.0, 1.0)
    assert pd.pd_plan_create(sp, 16, 0.1, 0.0, 0, 1.0, 1, None)[0] == pd.PD_ERR_ARG     # alpha = 0
    assert pd.pd_plan_create(sp, 16, 0.1, 1.5, 0, 1.0, 1, None)[0] == pd.PD_ERR_ARG     # alpha > 1
    assert pd.pd_plan_create(sp, 16, -0.1, 0.1, 0, 1.0, 1, None)[0] == pd.PD_ERR_ARG    # dt < 0
    # Nt = 5000 needs a Bluestein length of 16384 > 4096 rows
    assert pd.pd_plan_create(sp, 5000, 0.1, 0.1, 0, 1.0, 1, None)[0] == pd.PD_ERR_UNSUPPORTED
    assert pd.pd_plan_create(sp, 16, 0.1, 0.1, 7, 1.0, 1, None)[0] == pd.PD_ERR_ARG     # scheme
    sp2 = pd.pd_space(2, 15, 15, 0.1, 1.0, 0.0, 0, 0, 1.0, 1.0)   # Dirichlet x with advection
    assert pd.pd_plan_create(sp2, 16, 0.1, 0.1, 0, 1.0, 1, None)[0] == pd.PD_ERR_UNSUPPORTED
    sp3 = pd.pd_space(2, 15, 15, 0.1, 0.0, 0.0, 1, 1, 1.0, 1.0)   # periodic y
    assert pd.pd_plan_create(sp3, 16, 0.1, 0.1, 0, 1.0, 1, None)[0] == pd.PD_ERR_UNSUPPORTED


def test_pd1_plan_create_rejects_bad_arguments_without_gpu():
    import paradiag_gb300 as pd
    pd.build()
    sp = pd.pd_space(1, 15, 1, 0.1, 0.0, 0.0, 0, 0, 1.0, 1.0)
    assert pd.pd1_plan_create(sp, 0, 0.05, 1.2, 0, 1, 0, None)[0] == pd.PD_ERR_ARG       # nt
    assert pd.pd1_plan_create(sp, 40, 0.05, 1.2, 0, 1, 0, None)[0] == pd.PD_ERR_UNSUPPORTED
    assert pd.pd1_plan_create(sp, 16, 0.05, 1.0, 0, 1, 0, None)[0] == pd.PD_ERR_ARG      # tau
    assert pd.pd1_plan_create(sp, 16, -0.05, 1.2, 0, 1, 0, None)[0] == pd.PD_ERR_ARG     # dt
    assert pd.pd1_plan_create(sp, 16, 0.05, 1.2, 3, 1, 0, None)[0] == pd.PD_ERR_ARG      # scheme
    assert pd.pd1_plan_create(sp, 16, 0.05, 1.2, 0, 2, 0, None)[0] == pd.PD_ERR_ARG      # scaling
    sp2 = pd.pd_space(2, 15, 15, 0.1, 1.0, 0.0, 0, 0, 1.0, 1.0)   # Dirichlet x with advection
    assert pd.pd1_plan_create(sp2, 16, 0.05, 1.2, 0, 1, 0, None)[0] == pd.PD_ERR_UNSUPPORTED


def test_pdh_plan_create_rejects_bad_arguments_without_gpu():
    import paradiag_gb300 as pd
    pd.build()
    sp = pd.pd_space(1, 15, 1, 0.1, 0.0, 0.0, 0, 0, 1.0, 1.0)
    assert pd.pdh_plan_create(sp, 0, 0.01, 0, None)[0] == pd.PD_ERR_ARG          # nt
    assert pd.pdh_plan_create(sp, 5000, 0.01, 0, None)[0] == pd.PD_ERR_UNSUPPORTED
    assert pd.pdh_plan_create(sp, 16, 0.0, 0, None)[0] == pd.PD_ERR_ARG          # dt
    assert pd.pdh_plan_create(sp, 16, 0.01, 2, None)[0] == pd.PD_ERR_ARG         # precision


def test_pdc_plan_create_rejects_bad_arguments_without_gpu():
    import paradiag_gb300 as pd
    pd.build()
    sp = pd.pd_space(2, 15, 15, 1.0, 0.0, 0.0, 0, 0, 1.0, 1.0)
    assert pd.pdc_plan_create(sp, 2, 2.0, 1e-4, 0, None)[0] == pd.PD_ERR_ARG          # nt
    assert pd.pdc_plan_create(sp, 16, 2.0, 1e-4, 0, None)[0] == pd.PD_ERR_UNSUPPORTED  # 4 | nt
    assert pd.pdc_plan_create(sp, 17, 2.0, 0.0, 0, None)[0] == pd.PD_ERR_ARG          # gamma
    assert pd.pdc_plan_create(sp, 17, -1.0, 1e-4, 0, None)[0] == pd.PD_ERR_ARG        # T


def test_nonlinear_entry_points_reject_a_null_plan_without_gpu():
    import paradiag_gb300 as pd
    pd.build()
    assert pd.pd_nl_build_rhs(None, (0, 0, 1), None, None, None) == pd.PD_ERR_ARG
    assert pd.pd_nl_residual(None, (0, 0, 1), None, None, None)[0] == pd.PD_ERR_ARG
    assert pd.pd_nl_solve(None, (0, 0, 1), None, None, 1e-10, 10)[0] == pd.PD_ERR_ARG


def test_window_and_left_gmres_entry_points_reject_a_null_plan_without_gpu():
    import paradiag_gb300 as pd
    pd.build()
    assert pd.pd_nl_solve_windows(None, (0, 0, 1), None, None, 2, None, 1e-10, 10)[0] == \
        pd.PD_ERR_ARG
    assert pd.pdc_solve_left(None, None, None, 1e-7, 10, 20)[0] == pd.PD_ERR_ARG
