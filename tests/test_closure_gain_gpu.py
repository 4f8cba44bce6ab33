"""What the learned closure gains: trained on drag samples of resolved runs
(seeds 1-4), evaluated on a held-out seed against the resolved forces, the
network predicts the drag better than a Wen-Yu-form law fitted to the same
samples and better than the Stokes drag of the slip velocity."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_mlp_beats_fitted_correlation_on_held_out_seed():
    from paper_1011_2613_gb300 import closure as CL

    phis = (0.1, 0.3)
    x, t, seeds, _, cost = CL.drag_dataset(phis, seeds=(1, 2, 3, 4, 5), n=48, transient=300, every=40,
                                           snapshots=10)
    tr = np.isin(seeds, (1, 2, 3, 4))
    te = ~tr
    import torch

    trm = torch.tensor(tr, device=x.device)
    mlp, secs, loss = CL.train_closure(x[trm], t[trm], batch=1024, epochs=60, lr=1e-3)
    xte, tte = x[~trm], t[~trm].cpu().numpy()
    pred = mlp.predict(xte).cpu().numpy()
    e_mlp = CL.rel_error(pred, tte)
    wy = CL.wen_yu_fit(x[trm].cpu().numpy(), t[trm].cpu().numpy())
    e_wy = CL.rel_error(wy(xte.cpu().numpy()), tte)
    e_stokes = CL.rel_error(xte.cpu().numpy()[:, 1:4], tte)
    print(f"held-out relative error: mlp {e_mlp:.3f}, fitted Wen-Yu form {e_wy:.3f}, Stokes {e_stokes:.3f}; "
          f"{int(tr.sum())} train / {int(te.sum())} test samples")
    assert e_mlp < e_wy and e_mlp < e_stokes
