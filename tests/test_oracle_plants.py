"""Planted mistakes in the oracle, each caught by a pin.

The oracle's C source carries three switches that a separate build turns on
(-DOR_PLANT=k; the oracle itself is built with none):
  1  the first-order Dirichlet wall flux where the second-order one-sided
     formula of Sec. 3.3 applies;
  2  face-centre fluxes without their interpolation to the face centroid
     (Sec. 3.3);
  3  the right-hand side s instead of kappa s (the integral form integrates
     the source over the cut cell's volume);
  4  the two permittivities swapped where the boundary state of a dielectric
     interface is eliminated (Sec. 3.3.1, the matching condition);
  5  the first-order EB stencil divided by h instead of the ray length;
  6  the least-squares EB stencil with the boundary weight's sign dropped;
  7  the least-squares fit taken about the cell centre instead of the EB
     centroid;
  8  no unknown on a fluid fragment of zero volume (treated as covered);
  9  the Robin wall elimination with a2 entering with the wrong sign;
 10  the Helmholtz shift without the volume fraction;
 11  the Robin electrode elimination with the inward derivative taken as
     outward.
Each of 1-3 must make the single-phase quadratic-exactness pin fail, so that
pin does test the wall formula, the centroid interpolation and the volume
weighting; 4 must fail the multifluid exactness pin, the coaxial closed form and
the matching condition of the interface field; 5 must fail the linear exactness
of the first-order EB stencils, 6 and 7 that of the least-squares stencils; 8
must fail the quadratic exactness with an electrode surface on grid faces; 9
the quadratic exactness with Robin walls; 10 and 11 the quadratic exactness
with a Robin electrode on grid faces (10 through the zero-volume fragments,
whose rows must carry no shift), 11 also the second-order convergence on a
curved Robin electrode.
"""
import pytest

import oracle
import test_oracle_helmholtz as TH
import test_oracle_pins as T
import test_oracle_pins_3d as T3


@pytest.fixture
def plant(monkeypatch):
    def use(k):
        monkeypatch.setattr(oracle, "_lib", oracle.planted(k))
    return use


@pytest.mark.parametrize("k", [1, 2, 3])
def test_plant_breaks_quadratic_exactness(plant, k):
    plant(k)
    with pytest.raises(AssertionError):
        T.test_quadratic_exactness_single_phase(32, "circle")


def test_plant_without_centroid_interpolation_breaks_3d_planar_pin(plant):
    plant(2)
    with pytest.raises(AssertionError):
        T3.test_planar_electrode_truncation_zero(16)


def test_plant_with_swapped_permittivities_breaks_multifluid_pins(plant):
    plant(4)
    with pytest.raises(AssertionError):
        T.test_quadratic_exactness_multifluid(32)
    with pytest.raises(AssertionError):
        T.test_coaxial_closed_form_second_order(0.0)
    with pytest.raises(AssertionError):
        T.test_interface_field_satisfies_matching_condition(2)


def test_plant_in_first_order_eb_stencil_breaks_linear_exactness(plant):
    plant(5)
    for dim in (2, 3):
        with pytest.raises(AssertionError):
            T.test_linear_exactness_with_first_order_eb_stencils(dim)


@pytest.mark.parametrize("k", [6, 7])
@pytest.mark.parametrize("dim", [2, 3])
def test_plant_in_least_squares_stencil_breaks_linear_exactness(plant, k, dim):
    plant(k)
    with pytest.raises(AssertionError):
        T.test_linear_exactness_with_least_squares_eb_stencils(dim)


@pytest.mark.parametrize("dim", [2, 3])
def test_plant_without_zero_volume_unknowns_breaks_face_aligned_exactness(plant, dim):
    plant(8)
    with pytest.raises(AssertionError):
        T.test_quadratic_exactness_with_eb_on_grid_faces(dim, 0.0)


def test_unplanted_build_passes_the_same_pins():
    T.test_quadratic_exactness_single_phase(32, "circle")
    T3.test_planar_electrode_truncation_zero(16)
    T.test_quadratic_exactness_multifluid(32)
    T.test_interface_field_satisfies_matching_condition(2)
    T.test_linear_exactness_with_first_order_eb_stencils(2)
    T.test_linear_exactness_with_first_order_eb_stencils(3)
    for dim in (2, 3):
        T.test_linear_exactness_with_least_squares_eb_stencils(dim)
        T.test_quadratic_exactness_with_eb_on_grid_faces(dim, 0.0)


def test_plant_robin_wall_sign_breaks_robin_wall_exactness(plant):
    plant(9)
    for dim in (2, 3):
        with pytest.raises(AssertionError):
            TH.test_quadratic_exactness_with_robin_walls_and_helmholtz_shift(dim)


def test_plant_shift_without_volume_fraction_breaks_robin_electrode_exactness(plant):
    plant(10)
    with pytest.raises(AssertionError):
        TH.test_quadratic_exactness_with_robin_electrode_on_grid_faces(2, 0.0)


def test_plant_robin_electrode_direction_breaks_robin_electrode_pins(plant):
    plant(11)
    with pytest.raises(AssertionError):
        TH.test_quadratic_exactness_with_robin_electrode_on_grid_faces(2, 1e-10)
    with pytest.raises(AssertionError):
        TH.test_robin_disk_electrode_second_order()
