"""Failure detection on the GPU without a fault: the kernels' bounded waits,
made to run out on mbarriers that nothing completes, report SIL_ETIMEOUT and
pass the abort on, and the context stays usable afterwards.  Collected last:
it takes about a second of waiting by design."""
import numpy as np
import pytest
import torch

import oracle
from helpers import assert_scores, case, to_dev
from paper_2303_14102_gb300 import sil

pytestmark = pytest.mark.gpu


def test_waits_give_up_report_and_leave_the_context_usable():
    tc_bits, gather_bits, left_on_abort = sil.selftest_bounded_wait()
    assert tc_bits == sil.SIL_ETIMEOUT        # pass-2 wait: its limit, then SIL_ETIMEOUT
    assert gather_bits == sil.SIL_ETIMEOUT    # pass-1 wait: likewise
    assert left_on_abort == 1                 # a later wait left on the abort, before its own limit
    X, lab = case(9, 3000, 8, 5)
    Xt, lt = to_dev(X, lab)
    st = sil.new_status(Xt.device)
    r = sil.silhouette(Xt, lt, 5, want_s=True, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert_scores(r.s, r.S, oracle.linear(X.astype(np.float64), lab, 5))
