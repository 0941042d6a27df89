"""What the trained network gains over the method without it.

The MLP is trained on the GPU with the library's own forward, backward and
Adam kernels on seeded inclusion meshes (Young's modulus 10^U[-2,2] inside
random spheres), then the learned and the plain Chebyshev smoother are
compared on held-out instances by the convergence factor of the stationary
V-cycle iteration and by CG iterations to rtol 1e-8.  The plain smoother is
the fallback: the learned one is kept only if it converges faster on both
counts.  The test prints both forms' figures and checks that the decision
follows them; it does not require a gain."""
import json

import pytest
import torch

from paper_2606_24748_gb300 import bamg as B
from paper_2606_24748_gb300 import learned

pytestmark = pytest.mark.gpu


def test_learned_against_plain_on_held_out_meshes():
    B.lib()
    assert torch.cuda.is_available()
    res = learned.run(ne=16, n_train=40, n_test=8, epochs=8, log=print)
    summary = {k: res[k] for k in ("rho_plain", "rho_learned", "cg_its_plain", "cg_its_learned",
                                   "test_mse", "target_variance", "learned_better_fraction", "use_learned")}
    print("learned vs plain (16^3 inclusion meshes, 40 train / 8 held out):", json.dumps(summary))
    assert res["all_converged"]
    # both cycles contract once the first cycles' residual transient is left out
    assert 0.0 < res["rho_plain"] < 1.0 and 0.0 < res["rho_learned"] < 1.0
    # the network fits part of the targets' variance on unseen meshes
    assert res["test_mse"] < res["target_variance"]
    # the learned weights are in use in the learned runs
    assert any(abs(p["rho_learned"] - p["rho_plain"]) > 1e-9 for p in res["per_instance"])
    gain = res["rho_learned"] < res["rho_plain"] and res["cg_its_learned"] <= res["cg_its_plain"]
    assert res["use_learned"] == gain
