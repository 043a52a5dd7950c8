"""Seeded synthetic catalogs shared by the oracle, the tests and the benchmark.

This package only draws inputs (positions, weights, densities). It holds none of the
estimator's arithmetic: no painting, no Fourier transforms of the estimator, no binning.
"""
from .catalogs import (  # noqa: F401
    Catalog,
    SurveyGeometry,
    LognormalField,
    uniform_box,
    on_node_catalog,
    survey_geometry,
    lognormal_field,
    survey_catalog,
    survey_randoms,
    box_randoms,
    mock_batch_spec,
)
