"""Host logic of the pipeline that runs before any library call (CPU)."""
from types import SimpleNamespace

import pytest
import torch

from paper_2408_12282_gb300 import pipeline as PL


def test_multilight_refuses_stale_images_and_a_missing_output():
    """Host logic of the many-light renderer: the L1 upstream reads the
    per-(view, light) images, so a backward(target=...) after a weighted
    (env_w) forward, or before any forward, is refused; a weighted forward
    needs its output buffer. Both checks run before any library call."""
    fake = SimpleNamespace()
    with pytest.raises(ValueError, match="per-\\(view, light\\) images"):
        PL.MultiLightRenderer.backward(fake, target=torch.zeros(4, 3))
    fake._pair_images_current = False                 # as after forward(env_w=...)
    with pytest.raises(ValueError, match="per-\\(view, light\\) images"):
        PL.MultiLightRenderer.backward(fake, target=torch.zeros(4, 3))
    with pytest.raises(ValueError, match="out"):
        PL.MultiLightRenderer.forward(fake, env_w=torch.ones(2))
